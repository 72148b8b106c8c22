// Angular power spectrum, Eq. (APS), for real maps from the m >= 0 coefficients:
//     C_l = (|a_l^0|^2 + 2 sum_{m=1}^{l} |a_l^m|^2) / (2l + 1).
// A block covers 32 consecutive degrees of one map; its 8 warps split the orders
// m between them (warp w takes m = w, w+8, ...), so each load instruction reads
// 32 consecutive degrees at one m -- adjacent in the m-major packing.  All terms
// are positive, so plain sums lose at most n u of the total: a thread squares
// in the plan precision, adds groups of 4 squares in that precision and the
// group sums in double (for FP32 plans each group sum is within about 3e-7 of
// its exact value, and the double partial within about 1e-13); the 8 partials of a
// degree are then combined with Neumaier's compensated summation.  (Doing all
// of it in FP64 with compensation per term made this kernel FP64-bound on a
// GPU with low FP64 throughput.)
#include <algorithm>

#include "plan.h"

namespace hpx {

namespace {
__device__ __forceinline__ void neumaier(double& s, double& comp, double v) {
    const double t = s + v;
    if (fabs(s) >= fabs(v)) comp += (s - t) + v;
    else comp += (v - t) + s;
    s = t;
}
constexpr int kSlices = 8;
}  // namespace

// almoff / cloff / lmax: per-map element offsets and degrees of a concatenated
// uneven batch (one launch for all its maps), or NULL for a uniform batch.
template <class T>
__global__ void __launch_bounds__(32 * kSlices) cl_kernel(const cplx<T>* __restrict__ alm, double* __restrict__ cl,
                                                          int Lu, int64_t nalm, const int64_t* __restrict__ almoff,
                                                          const int64_t* __restrict__ cloff,
                                                          const int* __restrict__ lmax) {
    __shared__ double part[kSlices][32][2];
    const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
    const int l = blockIdx.x * 32 + lane;
    const int b = blockIdx.y;
    const int L = lmax ? lmax[b] : Lu;
    if (blockIdx.x * 32 > L) return;   // the whole block is past this map's degrees
    const cplx<T>* a = alm + (almoff ? almoff[b] : (int64_t)b * nalm);
    double s = 0.0;
    if (l <= L) {
        auto sq = [&](int m) {
            const cplx<T> v = a[(int64_t)m * (2 * L + 1 - m) / 2 + l];
            return v.r * v.r + v.i * v.i;
        };
        int m = slice;
        if (m == 0) {   // the m = 0 term has weight 1, all others 2
            s = (double)sq(0);
            m += kSlices;
        }
        double s2 = 0.0;
        for (; m + 3 * kSlices <= l; m += 4 * kSlices)
            s2 += (double)((sq(m) + sq(m + kSlices)) + (sq(m + 2 * kSlices) + sq(m + 3 * kSlices)));
        for (; m <= l; m += kSlices) s2 += (double)sq(m);
        s += 2.0 * s2;
    }
    part[slice][lane][0] = s;
    part[slice][lane][1] = 0.0;
    __syncthreads();
    if (slice == 0 && l <= L) {
        double S = 0.0, C = 0.0;
        for (int k = 0; k < kSlices; ++k) {
            neumaier(S, C, part[k][lane][0]);
            C += part[k][lane][1];
        }
        cl[(cloff ? cloff[b] : (int64_t)b * (L + 1)) + l] = (S + C) / (2.0 * l + 1.0);
    }
}

template <class T>
void launch_cl(const hpx_plan_s* P, const T* alm, double* cl, cudaStream_t s) {
    const auto& g = P->g;
    dim3 grid((g.L + 1 + 31) / 32, g.B);
    if (P->group)   // every map of an uneven batch in one launch, from the per-map tables
        cl_kernel<T><<<grid, 32 * kSlices, 0, s>>>((const cplx<T>*)alm, cl, g.L, g.nalm, P->d_almel, P->d_clel,
                                                   P->d_lmax);
    else
        cl_kernel<T><<<grid, 32 * kSlices, 0, s>>>((const cplx<T>*)alm, cl, g.L, g.nalm, nullptr, nullptr, nullptr);
}

// Vector-Jacobian product of Eq. (APS): for a loss L(C) with g_l = dL/dC_l, the
// gradient with respect to the packed coefficients (torch's convention for a
// complex input: dL/dRe a + i dL/dIm a) is
//     dL/da_lm = g_l 2 w_m a_lm / (2l + 1),   w_0 = 1, w_m = 2 (m > 0).
// One block per (order m, map b); the threads run over the degrees l = m..L_b.
// Maps are located through almoff / cloff (element offsets of map b's
// coefficients and spectrum) and lmax[b], so concatenated uneven batches work
// in place; a map with m > L_b has nothing to do for this block.
template <class T>
__global__ void __launch_bounds__(256) cl_vjp_kernel(const cplx<T>* __restrict__ alm, const double* __restrict__ gcl,
                                                     cplx<T>* __restrict__ galm, const int64_t* __restrict__ almoff,
                                                     const int64_t* __restrict__ cloff, const int* __restrict__ lmax,
                                                     int Lu, int64_t nalm_u) {
    const int m = blockIdx.x, b = blockIdx.y;
    const int L = lmax ? lmax[b] : Lu;
    if (m > L) return;
    const int64_t ao = almoff ? almoff[b] : (int64_t)b * nalm_u;
    const int64_t co = cloff ? cloff[b] : (int64_t)b * (Lu + 1);
    const int64_t i0 = ao + (int64_t)m * (2 * L + 1 - m) / 2;
    const double w = m == 0 ? 2.0 : 4.0;
    for (int l = m + threadIdx.x; l <= L; l += blockDim.x) {
        const T f = (T)(gcl[co + l] * w / (2.0 * l + 1.0));
        const cplx<T> a = alm[i0 + l];
        galm[i0 + l] = mk<T>(f * a.r, f * a.i);
    }
}

template <class T>
void launch_cl_vjp(const T* alm, const double* gcl, T* galm, const int64_t* almoff, const int64_t* cloff,
                   const int* lmax, int Lmax_all, int B, int Lu, int64_t nalm_u, cudaStream_t s) {
    dim3 grid(Lmax_all + 1, B);
    cl_vjp_kernel<T><<<grid, 256, 0, s>>>((const cplx<T>*)alm, gcl, (cplx<T>*)galm, almoff, cloff, lmax, Lu,
                                          nalm_u);
}

template void launch_cl_vjp<float>(const float*, const double*, float*, const int64_t*, const int64_t*, const int*,
                                   int, int, int, int64_t, cudaStream_t);
template void launch_cl_vjp<double>(const double*, const double*, double*, const int64_t*, const int64_t*,
                                    const int*, int, int, int, int64_t, cudaStream_t);

template <class T>
__global__ void finite_check_kernel(const T* __restrict__ x, int64_t n, int* __restrict__ status) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(x[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(status, HPX_ERR_NONFINITE);
}

void launch_finite_check(const void* x, int64_t n, bool fp64, int* status, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = std::max(1, std::min<int>(sms * 8, (int)((n + 255) / 256)));
    if (fp64) finite_check_kernel<double><<<blocks, 256, 0, s>>>((const double*)x, n, status);
    else finite_check_kernel<float><<<blocks, 256, 0, s>>>((const float*)x, n, status);
}

template void launch_cl<float>(const hpx_plan_s*, const float*, double*, cudaStream_t);
template void launch_cl<double>(const hpx_plan_s*, const double*, double*, cudaStream_t);

}  // namespace hpx
