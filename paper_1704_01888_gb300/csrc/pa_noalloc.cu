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
#include <mutex>

#include "../../include/pa.h"
#include "pa_internal.cuh"

namespace pa {

namespace {

// Limits of the fixed working memory.
constexpr int kMaxReplicas = 1 << 18;             // R_prev and parent capacity
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

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(unsigned char **out)
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
    *out = static_cast<unsigned char *>(g_scratch_ptr[dev]);
    return cudaSuccess;
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

}  // namespace

}  // namespace pa

extern "C" pa_status pa_resample_noalloc(const int32_t *E, int32_t R_prev, int32_t L, double dbeta, int32_t R_target,
                                         int32_t mode, int32_t step, uint64_t seed, int32_t *parent,
                                         int32_t parent_cap, double *lnQ_out, int32_t *R_out, void *cuda_stream)
{
    using namespace pa;
    if (!E || !parent || !lnQ_out || !R_out) return PA_ERR_INVALID;
    if (L < 2 || (L & 1) || R_prev < 1 || R_target < 1 || parent_cap < R_prev) return PA_ERR_INVALID;
    if (mode < PA_RESAMPLE_NEAREST_INT || mode > PA_RESAMPLE_OFF) return PA_ERR_INVALID;
    if (!(dbeta == dbeta) || dbeta > 1e300 || dbeta < -1e300) return PA_ERR_INVALID;
    if (L > kMaxL || R_prev > kMaxReplicas || parent_cap > kMaxReplicas) return PA_ERR_TOO_LARGE;

    unsigned char *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return PA_ERR_CUDA;
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
    k_na_clear<<<(nbins + 1023) / 1024, 1024, 0, s>>>(hist, nbins, st, R_prev);
    k_na_hist<<<(R_prev + 255) / 256, 256, 0, s>>>(E, R_prev, 2 * N, hist, st);
    bump_launch_count(2);
    cudaError_t e = launch_resample(hist, nbins, E, dbeta, R_target, parent_cap, mode, step, 0u, k0, k1, wtab, counts,
                                    local_off, blocksum, parent, hist, st, s);
    if (e != cudaSuccess) return PA_ERR_CUDA;
    k_na_outputs<<<1, 1, 0, s>>>(st, lnQ_out, R_out);
    bump_launch_count(1);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}
