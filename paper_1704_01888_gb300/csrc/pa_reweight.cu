// pa_reweight.cu -- the reweighting of population annealing as a function of
// the temperature step, with derivatives (Barash, Weigel, Shchur & Janke,
// arXiv:1704.01888, Sec. 2 step 2), and the adaptive temperature step.
//
//   ln Q(dbeta) = ln( sum_j exp(-dbeta E_j) / R ),  tau_j = exp(-dbeta E_j) / Q,
//   d ln Q / d dbeta = -<E>_tau,   d <E>_tau / d dbeta = -var_tau(E),
//   d var_tau(E) / d dbeta = -k3_tau(E),
//   <O>_tau = sum_j O_j tau_j / R,  d <O>_tau / d dbeta = -cov_tau(O, E),
//   d <O>_tau / d O_j = tau_j / R.
// The sums are taken about the reference energy E_ref (lowest energy for
// dbeta >= 0, highest otherwise) in a fixed order, with explicitly rounded
// double operations.
//
// Adaptive step (the paper uses constant steps; this is a reading added here):
// with mean-one weights t_j = R w_j / S, the overlap of the populations at
// beta and beta + dbeta is alpha = (1/R) sum_j min(1, t_j), with derivative
// alpha' = (1/R) sum_{t_j < 1} t_j (<E>_tau - E_j).  The step solves
// alpha = target by bisection-safeguarded Newton iterations, stopping once
// |alpha - target| <= 1e-12, and is rounded down to a multiple of 2^-24.
#include <climits>

#include "../../include/pa.h"
#include "pa_internal.cuh"

namespace pa {

namespace {

constexpr int kB = 1024;

// Fixed-order block sum; every thread receives the result.
__device__ double bsum(double v, double *sc)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xFFFFFFFFu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sc[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double r = (lane < (int)(blockDim.x >> 5)) ? sc[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = __dadd_rn(r, __shfl_down_sync(0xFFFFFFFFu, r, o));
        if (lane == 0) sc[0] = r;
    }
    __syncthreads();
    return sc[0];
}

// Block-wide min (lowest = true) or max of ints; every thread receives it.
__device__ int bextreme(int v, bool lowest, int *sc)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int w = __shfl_down_sync(0xFFFFFFFFu, v, o);
        v = lowest ? min(v, w) : max(v, w);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sc[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int r = (lane < (int)(blockDim.x >> 5)) ? sc[lane] : (lowest ? INT_MAX : INT_MIN);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int w = __shfl_down_sync(0xFFFFFFFFu, r, o);
            r = lowest ? min(r, w) : max(r, w);
        }
        if (lane == 0) sc[0] = r;
    }
    __syncthreads();
    return sc[0];
}

// out[0..7] = ln Q, <E>_tau, var_tau(E), <O>_tau, cov_tau(O, E), E_ref, S, k3_tau(E).
__global__ void __launch_bounds__(kB) k_rw_forward(const int32_t *E, const double *O, int R, const double *dbeta_p,
                                                   double *out)
{
    __shared__ double sd[32];
    __shared__ int si[32];
    const double dbeta = *dbeta_p;
    const bool lowest = dbeta >= 0.0;
    int ref = lowest ? INT_MAX : INT_MIN;
    for (int j = threadIdx.x; j < R; j += blockDim.x) ref = lowest ? min(ref, E[j]) : max(ref, E[j]);
    ref = bextreme(ref, lowest, si);
    double S = 0.0, S1 = 0.0, S2 = 0.0, S3 = 0.0, SO = 0.0, SOe = 0.0;
    for (int j = threadIdx.x; j < R; j += blockDim.x) {
        const double e = (double)(E[j] - ref);
        const double w = exp(__dmul_rn(-dbeta, e));
        const double we = __dmul_rn(w, e);
        const double wee = __dmul_rn(we, e);
        S = __dadd_rn(S, w);
        S1 = __dadd_rn(S1, we);
        S2 = __dadd_rn(S2, wee);
        S3 = __dadd_rn(S3, __dmul_rn(wee, e));
        if (O) {
            const double wo = __dmul_rn(w, O[j]);
            SO = __dadd_rn(SO, wo);
            SOe = __dadd_rn(SOe, __dmul_rn(wo, e));
        }
    }
    S = bsum(S, sd);
    S1 = bsum(S1, sd);
    S2 = bsum(S2, sd);
    S3 = bsum(S3, sd);
    if (O) {
        SO = bsum(SO, sd);
        SOe = bsum(SOe, sd);
    }
    if (threadIdx.x == 0) {
        const double m1 = __ddiv_rn(S1, S);
        const double m2 = __ddiv_rn(S2, S);
        const double m3 = __ddiv_rn(S3, S);
        out[0] = __dadd_rn(__dmul_rn(-dbeta, (double)ref), log(__ddiv_rn(S, (double)R)));
        out[1] = __dadd_rn((double)ref, m1);
        out[2] = __dsub_rn(m2, __dmul_rn(m1, m1));
        out[3] = O ? __ddiv_rn(SO, S) : 0.0;
        out[4] = O ? __dsub_rn(__ddiv_rn(SOe, S), __dmul_rn(__ddiv_rn(SO, S), m1)) : 0.0;
        out[5] = (double)ref;
        out[6] = S;
        out[7] = __dadd_rn(__dsub_rn(m3, __dmul_rn(__dmul_rn(3.0, m1), m2)),
                           __dmul_rn(__dmul_rn(__dmul_rn(2.0, m1), m1), m1));
    }
}

// dst[0] = sign * g[0] * src[idx]: the dbeta-gradient of one forward output.
__global__ void k_rw_scale(const double *src, int idx, double sign, const double *g, double *dst)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) dst[0] = __dmul_rn(__dmul_rn(sign, g[0]), src[idx]);
}

// grad_O[j] = g tau_j / R = g exp(-dbeta (E_j - E_ref)) / S.
__global__ void k_rw_grad_O(const int32_t *E, int R, const double *dbeta_p, const double *fwd, const double *g,
                            double *grad_O)
{
    const double dbeta = *dbeta_p;
    const double ref = fwd[5], S = fwd[6], gg = g[0];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < R; j += gridDim.x * blockDim.x) {
        const double w = exp(__dmul_rn(-dbeta, __dsub_rn((double)E[j], ref)));
        grad_O[j] = __dmul_rn(gg, __ddiv_rn(w, S));
    }
}

// Overlap and its derivative over the replicas: out[0..1] = alpha, alpha'.
__global__ void __launch_bounds__(kB) k_overlap(const int32_t *E, int R, const double *dbeta_p, double *out)
{
    __shared__ double sd[32];
    __shared__ int si[32];
    const double dbeta = *dbeta_p;
    const bool lowest = dbeta >= 0.0;
    int ref = lowest ? INT_MAX : INT_MIN;
    for (int j = threadIdx.x; j < R; j += blockDim.x) ref = lowest ? min(ref, E[j]) : max(ref, E[j]);
    ref = bextreme(ref, lowest, si);
    double S = 0.0, S1 = 0.0;
    for (int j = threadIdx.x; j < R; j += blockDim.x) {
        const double e = (double)(E[j] - ref);
        const double w = exp(__dmul_rn(-dbeta, e));
        S = __dadd_rn(S, w);
        S1 = __dadd_rn(S1, __dmul_rn(w, e));
    }
    S = bsum(S, sd);
    S1 = bsum(S1, sd);
    const double m1 = __ddiv_rn(S1, S);
    double a = 0.0, da = 0.0;
    for (int j = threadIdx.x; j < R; j += blockDim.x) {
        const double e = (double)(E[j] - ref);
        const double t = __ddiv_rn(__dmul_rn((double)R, exp(__dmul_rn(-dbeta, e))), S);
        if (t < 1.0) {
            a = __dadd_rn(a, t);
            da = __dadd_rn(da, __dmul_rn(t, __dsub_rn(m1, e)));
        } else {
            a = __dadd_rn(a, 1.0);
        }
    }
    a = bsum(a, sd);
    da = bsum(da, sd);
    if (threadIdx.x == 0) {
        out[0] = __ddiv_rn(a, (double)R);
        out[1] = __ddiv_rn(da, (double)R);
    }
}

// The overlap at x over an energy histogram (bins k, energies k - 2N).
__device__ void overlap_hist(const int32_t *hist, int nbins, int kref, double R, double x, double *sd, double *a_out,
                             double *da_out)
{
    double S = 0.0, S1 = 0.0;
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) {
        const int h = hist[k];
        if (h == 0) continue;
        const double e = (double)(k - kref);
        const double hw = __dmul_rn((double)h, exp(__dmul_rn(-x, e)));
        S = __dadd_rn(S, hw);
        S1 = __dadd_rn(S1, __dmul_rn(hw, e));
    }
    S = bsum(S, sd);
    S1 = bsum(S1, sd);
    const double m1 = __ddiv_rn(S1, S);
    double a = 0.0, da = 0.0;
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) {
        const int h = hist[k];
        if (h == 0) continue;
        const double e = (double)(k - kref);
        const double t = __ddiv_rn(__dmul_rn(R, exp(__dmul_rn(-x, e))), S);
        if (t < 1.0) {
            a = __dadd_rn(a, __dmul_rn((double)h, t));
            da = __dadd_rn(da, __dmul_rn((double)h, __dmul_rn(t, __dsub_rn(m1, e))));
        } else {
            a = __dadd_rn(a, (double)h);
        }
    }
    a = bsum(a, sd);
    da = bsum(da, sd);
    *a_out = __ddiv_rn(a, R);
    *da_out = __ddiv_rn(da, R);
}

// The Newton step on the current population's histogram (one block).
__global__ void __launch_bounds__(kB) k_newton_hist(const int32_t *hist, int nbins, const DevState *st, double target,
                                                    double cap, int iters, double *out)
{
    __shared__ double sd[32];
    __shared__ int si[32];
    int kref = INT_MAX;
    for (int k = threadIdx.x; k < nbins; k += blockDim.x)
        if (hist[k] > 0) kref = min(kref, k);
    kref = bextreme(kref, true, si);
    const double R = (double)st->pop;
    double a, da;
    overlap_hist(hist, nbins, kref, R, cap, sd, &a, &da);
    double x;
    if (a >= target) {
        x = cap;
    } else {
        double lo = 0.0, hi = cap;
        x = __dmul_rn(0.5, __dadd_rn(lo, hi));
        for (int it = 0; it < iters; ++it) {
            overlap_hist(hist, nbins, kref, R, x, sd, &a, &da);
            const double f = __dsub_rn(a, target);
            if (fabs(f) <= 1e-12) break;  // converged: stop before rounding noise decides the bracket
            if (f > 0.0) lo = x; else hi = x;
            double nx = da != 0.0 ? __dsub_rn(x, __ddiv_rn(f, da)) : __dmul_rn(0.5, __dadd_rn(lo, hi));
            if (!(nx > lo && nx < hi)) nx = __dmul_rn(0.5, __dadd_rn(lo, hi));
            x = nx;
        }
        const double qx = floor(__dmul_rn(x, 16777216.0)) / 16777216.0;
        x = qx > 0.0 ? qx : 1.0 / 16777216.0;
    }
    if (threadIdx.x == 0) {
        out[0] = x;
        out[1] = a;
    }
}

}  // namespace

cudaError_t launch_newton(const int32_t *hist, int nbins, const DevState *st, double target, double cap, int iters,
                          double *out, cudaStream_t s)
{
    k_newton_hist<<<1, kB, 0, s>>>(hist, nbins, st, target, cap, iters, out);
    bump_launch_count(1);
    return cudaGetLastError();
}

}  // namespace pa

extern "C" {

pa_status pa_reweight_forward(const int32_t *E, const double *O, int32_t R, const double *dbeta, double *out,
                              void *stream)
{
    if (!E || !dbeta || !out || R < 1) return PA_ERR_INVALID;
    pa::k_rw_forward<<<1, pa::kB, 0, (cudaStream_t)stream>>>(E, O, R, dbeta, out);
    pa::bump_launch_count(1);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

pa_status pa_reweight_scale(const double *src, int32_t idx, double sign, const double *g, double *dst, void *stream)
{
    if (!src || !g || !dst || idx < 0 || idx > 7) return PA_ERR_INVALID;
    pa::k_rw_scale<<<1, 32, 0, (cudaStream_t)stream>>>(src, idx, sign, g, dst);
    pa::bump_launch_count(1);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

pa_status pa_reweight_grad_O(const int32_t *E, int32_t R, const double *dbeta, const double *fwd, const double *g,
                             double *grad_O, void *stream)
{
    if (!E || !dbeta || !fwd || !g || !grad_O || R < 1) return PA_ERR_INVALID;
    int grid = (R + 255) / 256;
    if (grid > 4096) grid = 4096;
    pa::k_rw_grad_O<<<grid, 256, 0, (cudaStream_t)stream>>>(E, R, dbeta, fwd, g, grad_O);
    pa::bump_launch_count(1);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

pa_status pa_overlap(const int32_t *E, int32_t R, const double *dbeta, double *out, void *stream)
{
    if (!E || !dbeta || !out || R < 1) return PA_ERR_INVALID;
    pa::k_overlap<<<1, pa::kB, 0, (cudaStream_t)stream>>>(E, R, dbeta, out);
    pa::bump_launch_count(1);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

}  // extern "C"
