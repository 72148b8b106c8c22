// Angular power spectrum, Eq. (APS), for real maps from the m >= 0 coefficients:
//     C_l = (|a_l^0|^2 + 2 sum_{m=1}^{l} |a_l^m|^2) / (2l + 1).
// One thread per degree l (consecutive threads read consecutive l at fixed m,
// which are adjacent in the m-major packing); the sum is accumulated in FP64
// with Neumaier compensation, whatever the precision of the coefficients.
#include "plan.h"

namespace hpx {

template <class T>
__global__ void cl_kernel(const cplx<T>* __restrict__ alm, double* __restrict__ cl, int L, int64_t nalm) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (l > L) return;
    const cplx<T>* a = alm + (int64_t)b * nalm;
    double s = 0.0, comp = 0.0;
    for (int m = 0; m <= l; ++m) {
        const cplx<T> v = a[(int64_t)m * (2 * L + 1 - m) / 2 + l];
        const double re = (double)v.r, im = (double)v.i;
        const double term = (m == 0 ? 1.0 : 2.0) * (re * re + im * im);
        const double t = s + term;
        if (fabs(s) >= fabs(term)) comp += (s - t) + term;
        else comp += (term - t) + s;
        s = t;
    }
    cl[(int64_t)b * (L + 1) + l] = (s + comp) / (2.0 * l + 1.0);
}

template <class T>
void launch_cl(const hpx_plan_s* P, const T* alm, double* cl, cudaStream_t s) {
    const auto& g = P->g;
    dim3 grid((g.L + 1 + 127) / 128, g.B);
    cl_kernel<T><<<grid, 128, 0, s>>>((const cplx<T>*)alm, cl, g.L, g.nalm);
}

template void launch_cl<float>(const hpx_plan_s*, const float*, double*, cudaStream_t);
template void launch_cl<double>(const hpx_plan_s*, const double*, double*, cudaStream_t);

}  // namespace hpx
