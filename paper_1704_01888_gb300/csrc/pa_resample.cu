// pa_resample.cu -- initial populations, the resampling step and the
// per-step estimators of population annealing (Barash, Weigel, Shchur & Janke,
// arXiv:1704.01888).
//
//   k_init      Sec. 2 step 1 (uniform spins at beta_0 = 0) or Sec. 5 Eq. 6
//               (a uniformly chosen ground state per replica).
//   k_weights   Sec. 2 step 2: reference energy, Boltzmann factors
//               w_k = exp(-dbeta (E_k - E_ref)) per energy bin, their
//               histogram-weighted sum S and ln Q_i = -dbeta E_ref + ln(S/R_{i-1}).
//   k_counts    copy numbers r_j from rho_j = R w(E_j) / S and their
//               block-local exclusive scan (warp shuffles).
//   k_scatter   block offsets, the new population size R_i (checked against
//               the capacity) and the parent map parent[off_j + c] = j.
//   k_finalize  Sec. 2 step 4 / Sec. 3 Eq. 4: population averages from exact
//               integer sums, the fluctuation-formula specific heat, the
//               magnetisation of Eq. 5, ln Z of Eq. 2 and the family entropy.
// All floating-point steps that feed a decision (S, rho, the rounding test)
// use explicitly rounded operations so that no multiply-add is contracted.
#include <climits>

#include "pa_internal.cuh"

namespace pa {

namespace {

constexpr int kBlock = 1024;

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Fixed-order block sum of doubles (shuffle tree within warps, then across
// warp leaders); result valid in thread 0.
__device__ double block_sum_fixed(double v, double *scratch32)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xFFFFFFFFu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) scratch32[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = (lane < (int)(blockDim.x >> 5)) ? scratch32[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = __dadd_rn(r, __shfl_down_sync(0xFFFFFFFFu, r, o));
    }
    __syncthreads();
    return r;
}

__device__ long long block_sum_ll(long long v, long long *scratch32)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) scratch32[warp] = v;
    __syncthreads();
    long long r = 0;
    if (warp == 0) {
        r = (lane < (int)(blockDim.x >> 5)) ? scratch32[lane] : 0;
        r = warp_sum(r);
        if (lane == 0) scratch32[0] = r;
    }
    __syncthreads();
    r = scratch32[0];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
__global__ void k_init(uint8_t *spins, int32_t *anc, int q, int L, int R, uint32_t k0, uint32_t k1,
                       int ground)
{
    const int N = L * L;
    const int NH = N / 2;
    const int L2 = L / 2;
    const long long total = (long long)R * (N / 4);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int slot = (int)(i / (N / 4));
        const int quad = (int)(i - (long long)slot * (N / 4));
        uint8_t *rep = spins + (size_t)slot * N;
        uint8_t v[4];
        if (ground) {
            const uint4 w = philox10(make_uint4((uint32_t)slot >> 2, DOM_GROUND, 0u, 0u), k0, k1);
            const uint8_t alpha = (uint8_t)__umulhi(pick_word(w, slot & 3), (uint32_t)q);
            v[0] = v[1] = v[2] = v[3] = alpha;
        } else {
            const uint4 w = philox10(make_uint4((uint32_t)quad, DOM_INIT, 0u, (uint32_t)slot), k0, k1);
            v[0] = (uint8_t)__umulhi(w.x, (uint32_t)q);
            v[1] = (uint8_t)__umulhi(w.y, (uint32_t)q);
            v[2] = (uint8_t)__umulhi(w.z, (uint32_t)q);
            v[3] = (uint8_t)__umulhi(w.w, (uint32_t)q);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int site = 4 * quad + j;  // canonical y*L + x
            const int y = site / L, x = site - y * L;
            const int c = (x + y) & 1;
            rep[c * NH + y * L2 + (x >> 1)] = v[j];
        }
        if (quad == 0 && anc) anc[slot] = slot;
    }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_weights(const int32_t *hist, int nbins, double dbeta,
                                                    DevState *st, double *wtab)
{
    __shared__ double s_d[32];
    __shared__ long long s_l[32];
    if (st->err) return;
    const int tid = threadIdx.x;
    // reference bin: lowest occupied for dbeta >= 0, highest for dbeta < 0
    long long best = dbeta >= 0.0 ? (long long)INT_MAX : -1;
    for (int k = tid; k < nbins; k += blockDim.x) {
        if (hist[k] > 0) best = dbeta >= 0.0 ? min(best, (long long)k) : max(best, (long long)k);
    }
    // min/max through the sum helper's scratch: reduce by shuffles
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long other = __shfl_down_sync(0xFFFFFFFFu, best, o);
        best = dbeta >= 0.0 ? min(best, other) : max(best, other);
    }
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) s_l[warp] = best;
    __syncthreads();
    if (warp == 0) {
        long long v = (lane < (int)(blockDim.x >> 5)) ? s_l[lane] : (dbeta >= 0.0 ? (long long)INT_MAX : -1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long other = __shfl_down_sync(0xFFFFFFFFu, v, o);
            v = dbeta >= 0.0 ? min(v, other) : max(v, other);
        }
        if (lane == 0) s_l[0] = v;
    }
    __syncthreads();
    const int kref = (int)s_l[0];

    double part = 0.0;
    for (int k = tid; k < nbins; k += blockDim.x) {
        const double w = exp(__dmul_rn(-dbeta, (double)(k - kref)));
        wtab[k] = w;
        part = __dadd_rn(part, __dmul_rn((double)hist[k], w));
    }
    const double S = block_sum_fixed(part, s_d);
    if (tid == 0) {
        const int E_ref = kref - (nbins - 1);
        st->S = S;
        st->E_ref = E_ref;
        st->lnQ = __dadd_rn(__dmul_rn(-dbeta, (double)E_ref), log(S / (double)st->pop));
    }
}

// Block-wide exclusive scan of one int per thread; returns the exclusive
// prefix, writes the block total to *total.
__device__ int block_exclusive_scan(int v, int *scratch32, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scratch32[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = (lane < (int)(blockDim.x >> 5)) ? scratch32[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= o) s += y;
        }
        scratch32[lane] = s;  // inclusive prefix over warps
    }
    __syncthreads();
    const int before = (warp > 0 ? scratch32[warp - 1] : 0) + x - v;
    *total = scratch32[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kBlock) k_counts(const int32_t *E, int twoN, int R_target, int mode,
                                                   int step, uint32_t k0, uint32_t k1, const double *wtab,
                                                   int32_t *counts, int32_t *local_off, int32_t *blocksum,
                                                   DevState *st)
{
    __shared__ int s_i[32];
    if (st->err) return;
    const int R_prev = st->pop;
    if (blockIdx.x * blockDim.x >= (unsigned)R_prev) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    int r = 0;
    if (j < R_prev) {
        const double w = wtab[E[j] + twoN];
        const double rho = __ddiv_rn(__dmul_rn((double)R_target, w), st->S);
        const double n = floor(rho);
        const double frac = __dsub_rn(rho, n);
        int up;
        if (mode == 1) {
            up = frac >= 0.5;
        } else {
            const uint4 u = philox10(make_uint4((uint32_t)j >> 2, DOM_RESAMPLE, (uint32_t)step, 0u), k0, k1);
            up = (double)pick_word(u, j & 3) < __dmul_rn(frac, 4294967296.0);
        }
        r = (int)n + up;
        counts[j] = r;
    }
    int total;
    const int before = block_exclusive_scan(r, s_i, &total);
    if (j < R_prev) local_off[j] = before;
    if (threadIdx.x == 0) blocksum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kBlock) k_scatter(const int32_t *counts, const int32_t *local_off,
                                                    const int32_t *blocksum, int32_t *parent, int R_cap,
                                                    int32_t *hist_zero, int nbins, DevState *st)
{
    __shared__ long long s_l[32];
    if (st->err) return;
    const int R_prev = st->pop;
    const int nb = (R_prev + blockDim.x - 1) / blockDim.x;
    long long off = 0, tot = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const long long v = blocksum[b];
        tot += v;
        if (b < (int)blockIdx.x) off += v;
    }
    tot = block_sum_ll(tot, s_l);
    off = block_sum_ll(off, s_l);
    if (tot > R_cap || tot <= 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) st->err = 2;  // PA_ERR_CAPACITY
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st->pop_next = (int)tot;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nbins; k += gridDim.x * blockDim.x) hist_zero[k] = 0;
    if ((int)blockIdx.x >= nb) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < R_prev) {
        const int o = (int)off + local_off[j];
        const int r = counts[j];
        for (int c = 0; c < r; ++c) parent[o + c] = j;
    }
}

__global__ void __launch_bounds__(kBlock) k_finalize(DevState *st, unsigned long long *acc, int32_t *fam,
                                                     int R0, DevObs *obs, double beta, int q, int N,
                                                     int gathered, int resampled)
{
    __shared__ double s_d[32];
    __shared__ long long s_l[32];
    if (st->err) return;
    const int R = gathered ? st->pop_next : st->pop;
    double part = 0.0;
    long long nf = 0;
    if (fam) {
        for (int f = threadIdx.x; f < R0; f += blockDim.x) {
            const int c = fam[f];
            if (c > 0) {
                const double nu = (double)c / (double)R;
                part = __dsub_rn(part, __dmul_rn(nu, log(nu)));
                nf += 1;
                fam[f] = 0;
            }
        }
    }
    const double Sf = block_sum_fixed(part, s_d);
    nf = block_sum_ll(nf, s_l);
    if (threadIdx.x == 0) {
        const long long sE = (long long)acc[0], sE2 = (long long)acc[1], sM = (long long)acc[2];
        acc[0] = acc[1] = acc[2] = 0ull;
        const double meanE = (double)sE / (double)R;
        const double meanE2 = (double)sE2 / (double)R;
        const double C =
            __ddiv_rn(__dmul_rn(__dmul_rn(beta, beta), __dsub_rn(meanE2, __dmul_rn(meanE, meanE))), (double)N);
        const double meanM = (double)((long long)q * sM - (long long)N * R) / __dmul_rn((double)(q - 1), (double)R);
        double lnQ = 0.0;
        if (resampled) {
            lnQ = st->lnQ;
            st->lnZ = __dadd_rn(st->lnZ, lnQ);
        }
        if (gathered) {
            st->pop = R;
            st->parity ^= 1;
        }
        DevObs o;
        o.beta = beta;
        o.lnQ = lnQ;
        o.lnZ = st->lnZ;
        o.meanE = meanE;
        o.meanE2 = meanE2;
        o.C = C;
        o.meanM = meanM;
        o.S_f = fam ? Sf : 0.0;
        o.R = R;
        o.n_families = fam ? nf : 0;
        o.sumE = sE;
        o.sumE2 = sE2;
        o.sumMt = sM;
        *obs = o;
    }
}

__global__ void k_to_canonical(const uint8_t *spins, uint8_t *out, int L, long long count)
{
    const int N = L * L;
    const int NH = N / 2;
    const int L2 = L / 2;
    const long long total = count * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / N;
        const int site = (int)(i - r * N);
        const int y = site / L, x = site - y * L;
        const int c = (x + y) & 1;
        out[i] = spins[r * N + c * NH + y * L2 + (x >> 1)];
    }
}

int grid_for(long long work, int threads)
{
    long long g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 65535LL * 16) g = 65535LL * 16;
    return (int)g;
}

}  // namespace

cudaError_t launch_init(uint8_t *spins, int32_t *anc, int q, int L, int R, uint32_t k0, uint32_t k1,
                        int ground, cudaStream_t s)
{
    const long long work = (long long)R * (L * L / 4);
    k_init<<<grid_for(work, 256), 256, 0, s>>>(spins, anc, q, L, R, k0, k1, ground);
    bump_launch_count(1);
    return cudaGetLastError();
}

cudaError_t launch_resample(const int32_t *hist, int nbins, const int32_t *E, double dbeta, int R_target,
                            int R_cap, int mode, int step, uint32_t k0, uint32_t k1, double *wtab,
                            int32_t *counts, int32_t *local_off, int32_t *blocksum, int32_t *parent,
                            int32_t *hist_zero, DevState *st, cudaStream_t s)
{
    const int nb = (R_cap + kBlock - 1) / kBlock;
    k_weights<<<1, kBlock, 0, s>>>(hist, nbins, dbeta, st, wtab);
    k_counts<<<nb, kBlock, 0, s>>>(E, nbins - 1, R_target, mode, step, k0, k1, wtab, counts, local_off,
                                   blocksum, st);
    const int nb2 = nb > (nbins + kBlock - 1) / kBlock ? nb : (nbins + kBlock - 1) / kBlock;
    k_scatter<<<nb2, kBlock, 0, s>>>(counts, local_off, blocksum, parent, R_cap, hist_zero, nbins, st);
    bump_launch_count(3);
    return cudaGetLastError();
}

cudaError_t launch_finalize(DevState *st, unsigned long long *acc, int32_t *fam, int R0, DevObs *obs,
                            double beta, int q, int N, int gathered, int resampled, cudaStream_t s)
{
    k_finalize<<<1, kBlock, 0, s>>>(st, acc, fam, R0, obs, beta, q, N, gathered, resampled);
    bump_launch_count(1);
    return cudaGetLastError();
}

cudaError_t launch_to_canonical(const uint8_t *spins, uint8_t *out, int L, int64_t count, cudaStream_t s)
{
    k_to_canonical<<<grid_for(count * L * L, 256), 256, 0, s>>>(spins, out, L, count);
    bump_launch_count(1);
    return cudaGetLastError();
}

}  // namespace pa
