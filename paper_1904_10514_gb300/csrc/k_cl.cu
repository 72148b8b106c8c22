// Angular power spectrum, Eq. (APS), for real maps from the m >= 0 coefficients:
//     C_l = (|a_l^0|^2 + 2 sum_{m=1}^{l} |a_l^m|^2) / (2l + 1).
// A block covers 32 consecutive degrees of one map; its 8 warps split the orders
// m between them (warp w takes m = w, w+8, ...), so each load instruction reads
// 32 consecutive degrees at one m -- adjacent in the m-major packing.  Each
// partial sum is accumulated in FP64 with Neumaier compensation and the 8
// partials of a degree are combined the same way.
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

template <class T>
__global__ void __launch_bounds__(32 * kSlices) cl_kernel(const cplx<T>* __restrict__ alm, double* __restrict__ cl,
                                                          int L, int64_t nalm) {
    __shared__ double part[kSlices][32][2];
    const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
    const int l = blockIdx.x * 32 + lane;
    const int b = blockIdx.y;
    const cplx<T>* a = alm + (int64_t)b * nalm;
    double s = 0.0, comp = 0.0;
    if (l <= L) {
        for (int m = slice; m <= l; m += kSlices) {
            const cplx<T> v = a[(int64_t)m * (2 * L + 1 - m) / 2 + l];
            const double re = (double)v.r, im = (double)v.i;
            neumaier(s, comp, (m == 0 ? 1.0 : 2.0) * (re * re + im * im));
        }
    }
    part[slice][lane][0] = s;
    part[slice][lane][1] = comp;
    __syncthreads();
    if (slice == 0 && l <= L) {
        double S = 0.0, C = 0.0;
        for (int k = 0; k < kSlices; ++k) {
            neumaier(S, C, part[k][lane][0]);
            C += part[k][lane][1];
        }
        cl[(int64_t)b * (L + 1) + l] = (S + C) / (2.0 * l + 1.0);
    }
}

template <class T>
void launch_cl(const hpx_plan_s* P, const T* alm, double* cl, cudaStream_t s) {
    const auto& g = P->g;
    dim3 grid((g.L + 1 + 31) / 32, g.B);
    cl_kernel<T><<<grid, 32 * kSlices, 0, s>>>((const cplx<T>*)alm, cl, g.L, g.nalm);
}

template void launch_cl<float>(const hpx_plan_s*, const float*, double*, cudaStream_t);
template void launch_cl<double>(const hpx_plan_s*, const double*, double*, cudaStream_t);

}  // namespace hpx
