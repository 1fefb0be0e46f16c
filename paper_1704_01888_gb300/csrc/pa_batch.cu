// pa_batch.cu -- M independent population-annealing runs (Barash, Weigel,
// Shchur & Janke, arXiv:1704.01888, Sec. 2 steps 1-5), possibly with
// different q, L, R and schedules, advanced together: every temperature step
// is six or seven launches that each cover all runs (weights, copy numbers,
// parent map, a persistent sweep kernel over every run's replica groups -- one
// for the runs with q <= 16 and one for the others, pa_batch.cuh --,
// estimators, step counter).  Because the step index lives in device memory,
// one captured CUDA graph of a step is replayed for the whole schedule.
//
// The runs share one Philox key and differ by their stream numbers, so run m
// of a batch reproduces bit for bit a lone run (pa_init) with the same
// configuration; block shapes chosen by the autotuner never change results.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/pa.h"
#include "pa_batch.cuh"
#include "pa_trace.h"

namespace pa {

namespace {

__device__ __forceinline__ int run_of_chunk(const RunDev *runs, int M, int chunk)
{
    int lo = 0, hi = M - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (runs[mid].chunk0 <= chunk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_batch_init(const BatchArgs b)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < b.total_items;
         i += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = b.M - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (b.runs[mid].item0 <= i) lo = mid; else hi = mid - 1;
        }
        const RunDev &r = b.runs[lo];
        dev::init_item(r.buf[0], r.anc[0], r.q, r.L, i - r.item0, b.k0, b.k1, r.stream_hi, r.ground);
    }
}

__global__ void __launch_bounds__(kB) k_batch_weights(const BatchArgs b)
{
    __shared__ unsigned long long s_acc[dev::kSumLimbs];
    __shared__ long long s_l[32];
    const int m = blockIdx.x;
    const int i = *b.step_counter;
    const StepDev sp = b.steps[(size_t)i * b.M + m];
    if (!sp.active) return;
    const RunDev &r = b.runs[m];
    dev::weights_body(r.hist, r.nbins, sp.dbeta, sp.wtab, r.st, s_acc, s_l);
}

__global__ void __launch_bounds__(kB) k_batch_counts(const BatchArgs b)
{
    __shared__ int s_i[32];
    const int m = run_of_chunk(b.runs, b.M, blockIdx.x);
    const int i = *b.step_counter;
    const StepDev &sp = b.steps[(size_t)i * b.M + m];
    if (!sp.active) return;
    const RunDev &r = b.runs[m];
    dev::counts_body(blockIdx.x - r.chunk0, r.E, r.nbins - 1, r.R0, r.mode, i, r.stream_hi, b.k0, b.k1, sp.wtab,
                     r.counts, r.local_off, r.blocksum, r.st, s_i);
}

__global__ void __launch_bounds__(kB) k_batch_scatter(const BatchArgs b)
{
    __shared__ long long s_l[32];
    const int m = run_of_chunk(b.runs, b.M, blockIdx.x);
    const int i = *b.step_counter;
    if (!b.steps[(size_t)i * b.M + m].active) return;
    const RunDev &r = b.runs[m];
    dev::scatter_body(blockIdx.x - r.chunk0, r.nchunks, r.counts, r.local_off, r.blocksum, r.parent, r.R_cap, r.hist,
                      r.nbins, r.st, s_l);
}

__global__ void __launch_bounds__(kB) k_batch_finalize(const BatchArgs b)
{
    __shared__ double s_d[32];
    __shared__ long long s_l[32];
    const int m = blockIdx.x;
    const int i = *b.step_counter;
    const StepDev sp = b.steps[(size_t)i * b.M + m];
    if (!sp.active) return;
    const RunDev &r = b.runs[m];
    dev::finalize_body(r.st, r.acc, r.fam, r.R0, r.obs + i, sp.beta, r.q, r.N, b.gather, b.gather, s_d, s_l);
}

__global__ void k_batch_advance(int32_t *step_counter)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *step_counter += 1;
}

}  // namespace

}  // namespace pa

struct pa_batch {
    int M = 0, Kmax = 0;
    cudaStream_t stream = nullptr, capture_stream = nullptr;
    std::vector<pa_config> cfg;
    std::vector<int> K, theta, R_cap, rpb, nchunks;
    std::vector<pa::RunDev> runs_h;
    pa::RunDev *runs_d = nullptr;
    pa::StepDev *steps_d = nullptr;
    uint8_t *stage = nullptr;  // canonical-layout staging for pa_batch_get_spins
    size_t stage_bytes = 0;
    int32_t *counter_d = nullptr;
    int32_t *work_d = nullptr;   // 2 x (Kmax + 1) group counters of the sweep kernel's two parts
    int32_t *order_d = nullptr;  // run order of the sweep kernel's groups
    std::vector<void *> allocs;
    pa::BatchArgs args{};
    int smem_budget = 65536, threads = 512, grid = 0, sms = 0;
    bool has_part[2] = {false, false};  // runs with q <= 16 / q > 16
    int grid_part[2] = {0, 0};
    int n_parts = 0;
    bool ran = false;
};

namespace {

pa_status bfail(cudaError_t e)
{
    pa::record_cuda_error(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PA_ERR_NOMEM : PA_ERR_CUDA;
}

#define PB_CK(expr)                                        \
    do {                                                   \
        cudaError_t pb_e_ = (expr);                        \
        if (pb_e_ != cudaSuccess) return bfail(pb_e_);     \
    } while (0)

template <typename T>
pa_status balloc(pa_batch *b, T **p, size_t count)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return bfail(e);
    }
    b->allocs.push_back(*p);
    return PA_OK;
}

void batch_release(pa_batch *b)
{
    for (void *p : b->allocs) cudaFree(p);
    b->allocs.clear();
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    b->capture_stream = nullptr;
}

// The sweep kernel of part 0 (q <= 16, this file) or part 1 (q > 16).
pa::BatchSweepFn sweep_kernel(int part) { return part == 0 ? pa::k_batch_sweep<0> : pa::batch_sweep_kernel_hi(); }

// The sweep kernels of the parts the batch's runs need, one after the other.
void launch_sweeps(const pa_batch *b, const pa::BatchArgs &a, cudaStream_t s)
{
    for (int part = 0; part < 2; ++part)
        if (b->has_part[part]) sweep_kernel(part)<<<b->grid_part[part], b->threads, b->smem_budget, s>>>(a);
}

// Replicas per block for each run and the persistent grid for a shared-memory
// budget and a block size.
pa_status apply_launch(pa_batch *b, int budget, int threads)
{
    int dev = 0, optin = 0;
    PB_CK(cudaGetDevice(&dev));
    PB_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    if (budget < 1024 || threads < 64 || threads > 1024 || threads % 32) return PA_ERR_INVALID;
    for (int part = 0; part < 2; ++part) {
        if (!b->has_part[part]) continue;
        PB_CK(cudaFuncGetAttributes(&fa, sweep_kernel(part)));
        if (budget + (int)fa.sharedSizeBytes > optin) return PA_ERR_INVALID;
    }
    for (int m = 0; m < b->M; ++m) {
        const size_t padded = pa::replica_bytes(b->cfg[m].q, b->cfg[m].L);
        if (padded > (size_t)budget) return PA_ERR_INVALID;
        int r = (int)(budget / padded);
        if (r > b->cfg[m].R) r = b->cfg[m].R;
        if (r < 1) r = 1;
        b->rpb[m] = r;
        b->runs_h[m].rpb = r;
    }
    for (int part = 0; part < 2; ++part) {
        if (!b->has_part[part]) continue;
        const pa::BatchSweepFn k = sweep_kernel(part);
        PB_CK(cudaFuncGetAttributes(&fa, k));
        PB_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
        int per_sm = 0;
        PB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, (size_t)budget));
        if (per_sm < 1) return PA_ERR_INVALID;
        b->grid_part[part] = per_sm * b->sms;
    }
    b->smem_budget = budget;
    b->threads = threads;
    b->grid = b->grid_part[b->has_part[0] ? 0 : 1];
    // groups of the costliest runs first: cost ~ replicas x sites x sweeps x (4 + bits per state)
    std::vector<int32_t> order(b->M);
    std::vector<double> cost(b->M);
    for (int m = 0; m < b->M; ++m) {
        order[m] = m;
        const pa_config &g = b->cfg[m];
        cost[m] = (double)b->rpb[m] * g.L * g.L * std::max(b->theta[m], 1) * (4 + pa::state_bits(g.q));
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    PB_CK(cudaMemcpyAsync(b->order_d, order.data(), sizeof(int32_t) * b->M, cudaMemcpyHostToDevice, b->stream));
    PB_CK(cudaMemcpyAsync(b->runs_d, b->runs_h.data(), sizeof(pa::RunDev) * b->M, cudaMemcpyHostToDevice, b->stream));
    PB_CK(cudaStreamSynchronize(b->stream));
    return PA_OK;
}

// Enqueues the initial populations and their step-0 estimators.
pa_status enqueue_start(pa_batch *b)
{
    PB_CK(cudaMemsetAsync(b->counter_d, 0, sizeof(int32_t), b->stream));
    PB_CK(cudaMemsetAsync(b->work_d, 0, sizeof(int32_t) * 2 * (size_t)(b->Kmax + 1), b->stream));
    for (int m = 0; m < b->M; ++m) {
        const pa::RunDev &r = b->runs_h[m];
        pa::DevState h{};
        h.pop = b->cfg[m].R;
        h.lnZ = b->cfg[m].init_mode == PA_INIT_GROUND ? std::log((double)r.q) - b->cfg[m].beta0 * (double)(-2 * r.N)
                                                       : (double)r.N * std::log((double)r.q);
        PB_CK(cudaMemcpyAsync(r.st, &h, sizeof(h), cudaMemcpyHostToDevice, b->stream));
        PB_CK(cudaMemsetAsync(r.hist, 0, sizeof(int32_t) * r.nbins, b->stream));
        PB_CK(cudaMemsetAsync(r.acc, 0, sizeof(unsigned long long) * 3, b->stream));
        if (r.fam) PB_CK(cudaMemsetAsync(r.fam, 0, sizeof(int32_t) * r.R0, b->stream));
        PB_CK(cudaStreamSynchronize(b->stream));  // h lives on this stack frame
    }
    long long threads_total = (b->args.total_items + 255) / 256;
    int grid = (int)std::min<long long>(threads_total, 65535LL * 16);
    pa::k_batch_init<<<grid, 256, 0, b->stream>>>(b->args);
    pa::BatchArgs a0 = b->args;
    a0.gather = 0;
    launch_sweeps(b, a0, b->stream);
    pa::k_batch_finalize<<<b->M, pa::kB, 0, b->stream>>>(a0);
    pa::k_batch_advance<<<1, 1, 0, b->stream>>>(b->counter_d);
    pa::bump_launch_count(3 + b->n_parts);
    PB_CK(cudaGetLastError());
    return PA_OK;
}

// Enqueues one temperature step (the six launches).
pa_status enqueue_step(pa_batch *b, cudaStream_t s)
{
    pa::k_batch_weights<<<b->M, pa::kB, 0, s>>>(b->args);
    pa::k_batch_counts<<<b->args.total_chunks, pa::kB, 0, s>>>(b->args);
    pa::k_batch_scatter<<<b->args.total_chunks, pa::kB, 0, s>>>(b->args);
    launch_sweeps(b, b->args, s);
    pa::k_batch_finalize<<<b->M, pa::kB, 0, s>>>(b->args);
    pa::k_batch_advance<<<1, 1, 0, s>>>(b->counter_d);
    pa::bump_launch_count(5 + b->n_parts);
    PB_CK(cudaGetLastError());
    return PA_OK;
}

pa_status check_runs(const pa_batch *b)
{
    for (int m = 0; m < b->M; ++m) {
        pa::DevState h;
        PB_CK(cudaMemcpy(&h, b->runs_h[m].st, sizeof(h), cudaMemcpyDeviceToHost));
        if (h.err) return (pa_status)h.err;
    }
    return PA_OK;
}

std::mutex g_tune_mutex;
std::map<std::string, std::pair<int, int>> g_tune_cache;

// The GPU (name and SM count) and the batch's shape: the key of a tuned launch.
std::string tune_key(const pa_batch *b)
{
    std::string k;
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
        k += std::string(prop.name) + "/" + std::to_string(prop.multiProcessorCount) + "|";
    for (int m = 0; m < b->M; ++m)
        k += std::to_string(b->cfg[m].q) + "," + std::to_string(b->cfg[m].L) + "," + std::to_string(b->cfg[m].R) + "," +
             std::to_string(b->theta[m]) + ";";
    return k;
}

// Tuned launches kept across processes: the file named by PA_AUTOTUNE_CACHE
// (unset: none), one line per tuned shape, "key<TAB>budget<TAB>threads".
bool cache_file_lookup(const std::string &key, int *budget, int *threads)
{
    const char *path = std::getenv("PA_AUTOTUNE_CACHE");
    if (!path || !*path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    std::string line;
    bool found = false;
    int c;
    while (true) {
        line.clear();
        while ((c = std::fgetc(f)) != EOF && c != '\n') line.push_back((char)c);
        const size_t t1 = line.find('\t'), t2 = line.rfind('\t');
        if (t1 != std::string::npos && t2 != t1 && line.compare(0, t1, key) == 0 && t1 == key.size()) {
            *budget = std::atoi(line.c_str() + t1 + 1);
            *threads = std::atoi(line.c_str() + t2 + 1);
            found = *budget > 0 && *threads > 0;  // the last line for a key wins
        }
        if (c == EOF) break;
    }
    std::fclose(f);
    return found;
}

void cache_file_store(const std::string &key, int budget, int threads)
{
    const char *path = std::getenv("PA_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s\t%d\t%d\n", key.c_str(), budget, threads);
    std::fclose(f);
}

}  // namespace

extern "C" {

pa_status pa_batch_create(const pa_run_desc *runs, int32_t M, void *cuda_stream, pa_batch **out)
{
    pa::TraceRange trace("pa_batch_create");
    if (!out) return PA_ERR_INVALID;
    *out = nullptr;
    if (!runs || M < 1 || M > pa::kMaxRuns) return PA_ERR_INVALID;
    const uint64_t seed = runs[0].cfg.seed;
    for (int m = 0; m < M; ++m) {
        const pa_config &g = runs[m].cfg;
        if (g.q < 2 || g.q > 128 || g.L < 2 || g.L > 1024 || (g.L & 1) || g.R < 1 || g.stream < 0 ||
            g.stream > 255 || g.seed != seed || runs[m].K < 1 || runs[m].theta < 0 ||
            runs[m].theta > pa::kMaxTheta || !runs[m].betas)
            return PA_ERR_INVALID;
        if (g.resample_mode < PA_RESAMPLE_NEAREST_INT || g.resample_mode > PA_RESAMPLE_OFF) return PA_ERR_INVALID;
        if (g.init_mode != PA_INIT_RANDOM && g.init_mode != PA_INIT_GROUND) return PA_ERR_INVALID;
        if (!(g.beta0 >= 0.0) || runs[m].betas[0] != g.beta0) return PA_ERR_INVALID;
        if ((long long)g.L * g.L > pa::kMaxLatticeBytes) return PA_ERR_TOO_LARGE;
        for (int i = 0; i <= runs[m].K; ++i)
            if (!std::isfinite(runs[m].betas[i]) || !(runs[m].betas[i] >= 0.0)) return PA_ERR_INVALID;
    }
    pa_batch *b = new (std::nothrow) pa_batch();
    if (!b) return PA_ERR_NOMEM;
    auto fail = [&](pa_status e) {
        batch_release(b);
        delete b;
        return e;
    };
    b->M = M;
    b->stream = (cudaStream_t)cuda_stream;
    b->cfg.resize(M);
    b->K.resize(M);
    b->theta.resize(M);
    b->R_cap.resize(M);
    b->rpb.resize(M);
    b->nchunks.resize(M);
    b->runs_h.resize(M);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(bfail(e));

    pa_status s = PA_OK;
    int chunk0 = 0;
    size_t stage_bytes = 0;
    long long item0 = 0;
    for (int m = 0; m < M; ++m) {
        const pa_run_desc &d = runs[m];
        pa_config g = d.cfg;
        long long cap = g.R_cap > 0 ? g.R_cap : (long long)g.R + g.R / 4 + 1024;
        if (cap < g.R || cap >= (1LL << 24)) return fail(PA_ERR_INVALID);
        g.R_cap = (int32_t)cap;
        b->cfg[m] = g;
        b->K[m] = d.K;
        b->has_part[pa::batch_part(g.q)] = true;
        b->theta[m] = d.theta;
        b->Kmax = std::max(b->Kmax, d.K);
        pa::RunDev &r = b->runs_h[m];
        std::memset(&r, 0, sizeof(r));
        r.q = g.q;
        r.L = g.L;
        r.N = g.L * g.L;
        r.nbins = 2 * r.N + 1;
        r.R0 = g.R;
        r.R_cap = (int)cap;
        r.mode = g.resample_mode;
        r.K = d.K;
        r.ground = g.init_mode == PA_INIT_GROUND;
        r.stream_hi = (uint32_t)g.stream << 24;
        const int nc = std::max((r.R_cap + pa::kB - 1) / pa::kB, (r.nbins + pa::kB - 1) / pa::kB);
        r.chunk0 = chunk0;
        r.nchunks = nc;
        chunk0 += nc;
        b->nchunks[m] = nc;
        r.item0 = item0;
        item0 += (long long)g.R * (2 * pa::colour_words(g.L));
        const size_t spin_bytes = (size_t)r.R_cap * pa::replica_bytes(g.q, g.L);
        stage_bytes = std::max(stage_bytes, std::min((size_t)r.R_cap * r.N, (size_t)64 << 20));
        if ((s = balloc(b, &r.buf[0], spin_bytes)) || (s = balloc(b, &r.buf[1], spin_bytes)) ||
            (s = balloc(b, &r.E, r.R_cap)) || (s = balloc(b, &r.Mt, r.R_cap)) || (s = balloc(b, &r.hist, r.nbins)) ||
            (s = balloc(b, &r.counts, r.R_cap)) || (s = balloc(b, &r.local_off, r.R_cap)) ||
            (s = balloc(b, &r.blocksum, nc)) || (s = balloc(b, &r.parent, r.R_cap)) ||
            (s = balloc(b, &r.acc, 3)) || (s = balloc(b, &r.st, 1)) ||
            (s = balloc(b, &r.obs, (size_t)d.K + 1)))
            return fail(s);
        if (g.track_families) {
            if ((s = balloc(b, &r.anc[0], r.R_cap)) || (s = balloc(b, &r.anc[1], r.R_cap)) ||
                (s = balloc(b, &r.fam, g.R)))
                return fail(s);
        }
    }
    b->n_parts = (int)b->has_part[0] + (int)b->has_part[1];
    // weight tables: one per run and distinct dbeta of its schedule (a
    // constant schedule has a handful), all in one device array
    std::vector<std::map<uint64_t, size_t>> wt_at(M);
    size_t wt_total = 0;
    for (int m = 0; m < M; ++m) {
        for (int i = 1; i <= b->K[m]; ++i) {
            const double dbeta = runs[m].betas[i] - runs[m].betas[i - 1];
            uint64_t key;
            std::memcpy(&key, &dbeta, sizeof(key));
            if (wt_at[m].emplace(key, wt_total).second) wt_total += (size_t)b->runs_h[m].nbins;
        }
    }
    std::vector<double> wt_host(wt_total);
    for (int m = 0; m < M; ++m) {
        for (const auto &kv : wt_at[m]) {
            double dbeta;
            std::memcpy(&dbeta, &kv.first, sizeof(dbeta));
            pa::weight_table(dbeta, b->runs_h[m].nbins, wt_host.data() + kv.second);
        }
    }
    double *wt_dev = nullptr;
    if ((s = balloc(b, &wt_dev, wt_total))) return fail(s);
    e = cudaMemcpy(wt_dev, wt_host.data(), sizeof(double) * wt_total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(bfail(e));
    // per-step parameters (step 0 = the initial measurement)
    std::vector<pa::StepDev> steps((size_t)(b->Kmax + 1) * M);
    for (int i = 0; i <= b->Kmax; ++i) {
        for (int m = 0; m < M; ++m) {
            pa::StepDev &sp = steps[(size_t)i * M + m];
            std::memset(&sp, 0, sizeof(sp));
            sp.active = i <= b->K[m];
            if (!sp.active) continue;
            const double beta = runs[m].betas[i];
            sp.beta = beta;
            sp.dbeta = i > 0 ? beta - runs[m].betas[i - 1] : 0.0;
            if (i > 0) {
                uint64_t key;
                std::memcpy(&key, &sp.dbeta, sizeof(key));
                sp.wtab = wt_dev + wt_at[m].at(key);
            }
            sp.theta = i > 0 ? b->theta[m] : 0;
            sp.thr = pa::acceptance_thresholds(beta);
        }
    }
    if ((s = balloc(b, &b->runs_d, M)) || (s = balloc(b, &b->steps_d, steps.size())) ||
        (s = balloc(b, &b->counter_d, 1)) || (s = balloc(b, &b->work_d, 2 * ((size_t)b->Kmax + 1))) ||
        (s = balloc(b, &b->order_d, M)))
        return fail(s);
    e = cudaMemcpy(b->steps_d, steps.data(), sizeof(pa::StepDev) * steps.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(bfail(e));

    pa::BatchArgs &a = b->args;
    a.steps = b->steps_d;
    a.runs = b->runs_d;
    a.step_counter = b->counter_d;
    a.work = b->work_d;
    a.work_stride = b->Kmax + 1;
    a.order = b->order_d;
    a.M = M;
    a.total_chunks = chunk0;
    a.total_items = item0;
    a.k0 = (uint32_t)(seed & 0xFFFFFFFFu);
    a.k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        a.rk0[r] = a.k0 + 0x9E3779B9u * (uint32_t)r;
        a.rk1[r] = a.k1 + 0xBB67AE85u * (uint32_t)r;
    }
    a.gather = 1;
    int budget = 65536;
    for (int m = 0; m < M; ++m) budget = std::max(budget, (int)pa::replica_bytes(b->cfg[m].q, b->cfg[m].L));
    if ((s = balloc(b, &b->stage, stage_bytes))) return fail(s);
    b->stage_bytes = stage_bytes;
    if ((s = apply_launch(b, budget, 512))) return fail(s);
    if ((s = enqueue_start(b))) return fail(s);
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return fail(bfail(e));
    if ((s = check_runs(b))) return fail(s);
    *out = b;
    return PA_OK;
}

pa_status pa_batch_set_launch(pa_batch *b, int32_t smem_budget, int32_t threads)
{
    if (!b) return PA_ERR_INVALID;
    if (b->ran) return PA_ERR_STATE;
    return apply_launch(b, smem_budget, threads);
}

pa_status pa_batch_get_launch(pa_batch *b, int32_t *smem_budget, int32_t *threads, int32_t *blocks)
{
    if (!b) return PA_ERR_INVALID;
    if (smem_budget) *smem_budget = b->smem_budget;
    if (threads) *threads = b->threads;
    if (blocks) *blocks = b->grid;
    return PA_OK;
}

pa_status pa_batch_run(pa_batch *b, int32_t use_graph)
{
    pa::TraceRange trace("pa_batch_run");
    if (!b) return PA_ERR_INVALID;
    if (b->ran) return PA_ERR_STATE;
    b->ran = true;
    if (!use_graph) {
        for (int i = 1; i <= b->Kmax; ++i) {
            pa_status s = enqueue_step(b, b->stream);
            if (s) return s;
        }
    } else {
        if (!b->capture_stream) PB_CK(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        PB_CK(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
        pa_status s = enqueue_step(b, b->capture_stream);
        cudaError_t e = cudaStreamEndCapture(b->capture_stream, &graph);
        if (s) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        for (int i = 1; i <= b->Kmax && e == cudaSuccess; ++i) e = cudaGraphLaunch(exec, b->stream);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bfail(e);
        pa::bump_launch_count((5LL + b->n_parts) * (b->Kmax - 1));
    }
    PB_CK(cudaStreamSynchronize(b->stream));
    return check_runs(b);
}

pa_status pa_batch_observables(pa_batch *b, int32_t m, pa_obs *out)
{
    if (!b || !out || m < 0 || m >= b->M) return PA_ERR_INVALID;
    PB_CK(cudaStreamSynchronize(b->stream));
    static_assert(sizeof(pa::DevObs) == sizeof(pa_obs), "pa_obs layout");
    PB_CK(cudaMemcpy(out, b->runs_h[m].obs, sizeof(pa_obs) * (size_t)(b->K[m] + 1), cudaMemcpyDeviceToHost));
    return PA_OK;
}

pa_status pa_batch_get_spins(pa_batch *b, int32_t m, int64_t slot_begin, int64_t count, uint8_t *host)
{
    if (!b || !host || m < 0 || m >= b->M || slot_begin < 0 || count < 0) return PA_ERR_INVALID;
    PB_CK(cudaStreamSynchronize(b->stream));
    const pa::RunDev &r = b->runs_h[m];
    pa::DevState h;
    PB_CK(cudaMemcpy(&h, r.st, sizeof(h), cudaMemcpyDeviceToHost));
    if (slot_begin + count > h.pop) return PA_ERR_INVALID;
    if (count == 0) return PA_OK;
    const size_t RW = (size_t)pa::replica_words(r.q, r.L);
    const int64_t per = (int64_t)(b->stage_bytes / (size_t)r.N);
    for (int64_t done = 0; done < count; done += per) {
        const int64_t n = count - done < per ? count - done : per;
        PB_CK(pa::launch_to_canonical(r.buf[h.parity] + (size_t)(slot_begin + done) * RW, b->stage, r.q, r.L, n,
                                      b->stream));
        PB_CK(cudaMemcpyAsync(host + (size_t)done * r.N, b->stage, (size_t)n * r.N, cudaMemcpyDeviceToHost,
                              b->stream));
        PB_CK(cudaStreamSynchronize(b->stream));
    }
    return PA_OK;
}

pa_status pa_batch_autotune(pa_batch *b, int32_t *smem_budget_out, int32_t *threads_out)
{
    pa::TraceRange trace("pa_batch_autotune");
    if (!b) return PA_ERR_INVALID;
    if (b->ran) return PA_ERR_STATE;
    const std::string key = tune_key(b);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        int cb = 0, ct = 0;
        if (it == g_tune_cache.end() && cache_file_lookup(key, &cb, &ct)) it = g_tune_cache.emplace(key, std::make_pair(cb, ct)).first;
        if (it != g_tune_cache.end()) {
            pa_status s = apply_launch(b, it->second.first, it->second.second);
            if (s) return s;
            if (smem_budget_out) *smem_budget_out = b->smem_budget;
            if (threads_out) *threads_out = b->threads;
            return PA_OK;
        }
    }
    // Each candidate times the first kTuneSteps temperature steps from the same
    // initial populations (restarted between candidates); shapes never change
    // results.
    constexpr int kTuneSteps = 3;
    const int tune_steps = std::min(kTuneSteps, b->Kmax);
    const int budgets[] = {32768, 49152, 65536, 98304, 131072};
    const int thread_opts[] = {256, 512, 1024};
    cudaEvent_t e0, e1;
    PB_CK(cudaEventCreate(&e0));
    PB_CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int best_budget = b->smem_budget, best_threads = b->threads;
    for (int budget : budgets) {
        for (int threads : thread_opts) {
            if (apply_launch(b, budget, threads) != PA_OK) continue;
            pa_status s = enqueue_start(b);
            if (s) return s;
            PB_CK(cudaEventRecord(e0, b->stream));
            for (int k = 0; k < tune_steps; ++k)
                if ((s = enqueue_step(b, b->stream))) return s;
            PB_CK(cudaEventRecord(e1, b->stream));
            PB_CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            PB_CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) {
                best_ms = ms;
                best_budget = budget;
                best_threads = threads;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pa_status s = apply_launch(b, best_budget, best_threads);
    if (s) return s;
    if ((s = enqueue_start(b))) return s;  // restart from the initial populations
    PB_CK(cudaStreamSynchronize(b->stream));
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = {best_budget, best_threads};
        cache_file_store(key, best_budget, best_threads);
    }
    if (smem_budget_out) *smem_budget_out = best_budget;
    if (threads_out) *threads_out = best_threads;
    return check_runs(b);
}

pa_status pa_batch_population_size(pa_batch *b, int32_t m, int32_t *R_out)
{
    if (!b || !R_out || m < 0 || m >= b->M) return PA_ERR_INVALID;
    PB_CK(cudaStreamSynchronize(b->stream));
    pa::DevState h;
    PB_CK(cudaMemcpy(&h, b->runs_h[m].st, sizeof(h), cudaMemcpyDeviceToHost));
    *R_out = h.pop;
    return h.err ? (pa_status)h.err : PA_OK;
}

pa_status pa_batch_measurements(pa_batch *b, int32_t m, int32_t *E_out, int32_t *Mt_out)
{
    if (!b || m < 0 || m >= b->M) return PA_ERR_INVALID;
    PB_CK(cudaStreamSynchronize(b->stream));
    const pa::RunDev &r = b->runs_h[m];
    pa::DevState h;
    PB_CK(cudaMemcpy(&h, r.st, sizeof(h), cudaMemcpyDeviceToHost));
    if (E_out) PB_CK(cudaMemcpy(E_out, r.E, sizeof(int32_t) * h.pop, cudaMemcpyDeviceToHost));
    if (Mt_out) PB_CK(cudaMemcpy(Mt_out, r.Mt, sizeof(int32_t) * h.pop, cudaMemcpyDeviceToHost));
    return h.err ? (pa_status)h.err : PA_OK;
}

void pa_batch_destroy(pa_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_release(b);
    delete b;
}

}  // extern "C"
