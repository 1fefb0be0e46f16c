// pa_noalloc.cu -- a resampling entry point that allocates no device memory.
//
// pa_resample_noalloc() runs the same resampling kernels as pa_resample(), but
// on caller-owned arrays (energies in, parent map out) and with its working
// memory taken from one fixed array in the library's own device image
// instead of cudaMalloc.  It serves callers that may not allocate: plug-ins
// whose host framework owns every device allocation (memory taken behind its
// back escapes its accounting and limits), and runtimes that must not touch
// the allocator once they are set up (an allocation can synchronise the device
// or fail under memory pressure in the middle of their work).
//
// The array is a file-scope __device__ variable, so every GPU that loads this
// library holds it (kScratchBytes, about 3.6 MB) until the process exits.
// Host code cannot use the variable's name as a device address: the first call
// on each device looks the address up with cudaGetSymbolAddress (with that
// device current) and caches it, and every launch receives that pointer.
// All calls share the one array and each call overwrites it, so calls whose
// work overlaps on the GPU (different streams without ordering between them)
// race; calls on one stream, or otherwise ordered, are safe.
//
// The Boltzmann factors come from the same host table as pa_resample's
// (pa::weight_table, the C library's exp), so both calls give the same copy
// numbers bit for bit.  The table is copied from a static host buffer into the
// fixed array; a call with the dbeta of the previous call on that device
// reuses it.
#include <cstring>
#include <mutex>

#include "../../include/pa.h"
#include "pa_internal.cuh"

namespace pa {

namespace {

// Limits of the fixed working memory.
constexpr int kMaxReplicas = 1 << 18;             // R_prev
constexpr int kMaxL = 256;                        // lattice size (2N + 1 energy bins)
constexpr int kMaxBins = 2 * kMaxL * kMaxL + 1;
constexpr int kMaxBlocks = (kMaxReplicas + 1023) / 1024;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffState = 0;
constexpr size_t kOffHist = align256(kOffState + sizeof(DevState));
constexpr size_t kOffWtab = align256(kOffHist + sizeof(int32_t) * kMaxBins);
constexpr size_t kOffCounts = align256(kOffWtab + sizeof(double) * kMaxBins);
constexpr size_t kOffLocal = align256(kOffCounts + sizeof(int32_t) * kMaxReplicas);
constexpr size_t kOffBlocks = align256(kOffLocal + sizeof(int32_t) * kMaxReplicas);
constexpr size_t kScratchBytes = align256(kOffBlocks + sizeof(int32_t) * kMaxBlocks);

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};
// the weight table held in each device's array: dbeta's bits and its length
uint64_t g_wtab_key[kMaxDevices] = {};
int g_wtab_len[kMaxDevices] = {};
double g_wtab_host[kMaxBins];  // host staging of the table (under g_setup_mutex)

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(int *dev_out, unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *dev_out = dev;
    *out = static_cast<unsigned char *>(g_scratch_ptr[dev]);
    return cudaSuccess;
}

// Loads the weight table of dbeta (nbins entries) into the device's array
// unless it already holds it.
cudaError_t load_wtab(int dev, double *wtab, double dbeta, int nbins, cudaStream_t s)
{
    uint64_t key;
    std::memcpy(&key, &dbeta, sizeof(key));
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_wtab_len[dev] >= nbins && g_wtab_key[dev] == key) return cudaSuccess;
    weight_table(dbeta, nbins, g_wtab_host);
    // from pageable memory: the call returns once the table has left the
    // static buffer, which the next call may then overwrite
    const cudaError_t e = cudaMemcpyAsync(wtab, g_wtab_host, sizeof(double) * (size_t)nbins,
                                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        g_wtab_key[dev] = key;
        g_wtab_len[dev] = nbins;
    } else {
        g_wtab_len[dev] = 0;
    }
    return e;
}

// Clears the histogram and sets the run state for one call.
__global__ void k_na_clear(int32_t *hist, int nbins, DevState *st, int R_prev)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nbins; k += gridDim.x * blockDim.x) hist[k] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        DevState s{};
        s.pop = R_prev;
        *st = s;
    }
}

// Energy histogram, bin E + 2N; an energy outside [-2N, 0] flags the call.
__global__ void k_na_hist(const int32_t *E, int R_prev, int twoN, int32_t *hist, DevState *st)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < R_prev; j += gridDim.x * blockDim.x) {
        const int e = E[j];
        if (e < -twoN || e > 0) {
            atomicExch(&st->err, (int)PA_ERR_INVALID);
        } else {
            atomicAdd(hist + (e + twoN), 1);
        }
    }
}

__global__ void k_na_outputs(const DevState *st, double *lnQ_out, int32_t *R_out)
{
    if (st->err) {
        *R_out = -st->err;
        *lnQ_out = 0.0;
    } else {
        *R_out = st->pop_next;
        *lnQ_out = st->lnQ;
    }
}

pa_status launch_failed(cudaError_t e)
{
    record_cuda_error(cudaGetErrorString(e));
    return PA_ERR_CUDA;
}

}  // namespace

}  // namespace pa

extern "C" pa_status pa_resample_noalloc(const int32_t *E, int32_t R_prev, int32_t L, double dbeta, int32_t R_target,
                                         int32_t mode, int32_t step, uint64_t seed, int32_t rng_stream,
                                         int32_t *parent, int32_t parent_cap, double *lnQ_out, int32_t *R_out,
                                         void *cuda_stream)
{
    using namespace pa;
    if (!E || !parent || !lnQ_out || !R_out) return PA_ERR_INVALID;
    if (L < 2 || (L & 1) || R_prev < 1 || R_target < 1 || parent_cap < R_prev) return PA_ERR_INVALID;
    if (mode < PA_RESAMPLE_NEAREST_INT || mode > PA_RESAMPLE_OFF) return PA_ERR_INVALID;
    if (rng_stream < 0 || rng_stream > 255) return PA_ERR_INVALID;
    if (!(dbeta == dbeta) || dbeta > 1e300 || dbeta < -1e300) return PA_ERR_INVALID;
    if (L > kMaxL || R_prev > kMaxReplicas) return PA_ERR_TOO_LARGE;
    // an error left pending by earlier work on this thread stays the caller's:
    // refuse to run rather than report it as ours or clear it
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) {
        record_cuda_error(cudaGetErrorString(pending));
        return PA_ERR_CUDA;
    }

    int dev = 0;
    unsigned char *base = nullptr;
    cudaError_t e = scratch_address(&dev, &base);
    if (e != cudaSuccess) return launch_failed(e);
    DevState *st = reinterpret_cast<DevState *>(base + kOffState);
    int32_t *hist = reinterpret_cast<int32_t *>(base + kOffHist);
    double *wtab = reinterpret_cast<double *>(base + kOffWtab);
    int32_t *counts = reinterpret_cast<int32_t *>(base + kOffCounts);
    int32_t *local_off = reinterpret_cast<int32_t *>(base + kOffLocal);
    int32_t *blocksum = reinterpret_cast<int32_t *>(base + kOffBlocks);

    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int N = L * L;
    const int nbins = 2 * N + 1;
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
    if ((e = load_wtab(dev, wtab, dbeta, nbins, s)) != cudaSuccess) return launch_failed(e);
    k_na_clear<<<(nbins + 1023) / 1024, 1024, 0, s>>>(hist, nbins, st, R_prev);
    bump_launch_count(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return launch_failed(e);
    k_na_hist<<<(R_prev + 255) / 256, 256, 0, s>>>(E, R_prev, 2 * N, hist, st);
    bump_launch_count(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return launch_failed(e);
    e = launch_resample(hist, nbins, E, dbeta, R_target, parent_cap, mode, step, (uint32_t)rng_stream << 24, k0, k1,
                        wtab, counts, local_off, blocksum, parent, hist, st, s);
    if (e != cudaSuccess) return launch_failed(e);
    k_na_outputs<<<1, 1, 0, s>>>(st, lnQ_out, R_out);
    bump_launch_count(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return launch_failed(e);
    return PA_OK;
}
