// The HEALPix software's analysis (Sec. 2.2), on the GPU: the equal-weight
// quadrature of Eq. (healsph),
//     a_l^m = (4 pi / N) sum_i conj(Y_l^m(x_i)) f(x_i),
// and its Jacobi (Richardson) refinement of Eqs. (uzawa) / (richardson),
//     a^(0) = A f,  a^(k+1) = a^(k) + A (f - S a^(k)),   A = (4 pi / N) S^*,
// where S is the spherical-harmonic synthesis of Eq. (synthesis)
// (hpx_sh_synthesis).  The paper's comparison method for HP2SPH.
//
// S^* f is the transpose of the synthesis under the library's real inner
// products (maps: sum_i f_i g_i; coefficients: weight 2 for m > 0), i.e. every
// stage of the synthesis transposed in reverse order:
//   ring stage     for every ring pair the DFT of the packed samples and, for each
//                  m <= lmax, the Fourier sum sum_k f_k e^{-i m lambda_k} (m mod
//                  nphi: the polar rings alias) with the synthesis' fold weights
//                  (launch_ring_fft with ew != 0); the pole rows are zero (no
//                  pixel sits at a pole);
//   NUFFT          the transpose of the synthesis' type-2 NUFFT: the analysis'
//                  type-1 NUFFT (spreading + grid FFT);
//   Legendre       the transpose of the synthesis' order-m -> latitude-Fourier
//                  conversion: its operators R_{m,c} Es applied row-wise (the
//                  per-order operator kernel on synM), or Es applied by the dense
//                  kernel followed by the forward Givens sweeps.
#include "plan.h"

namespace hpx {

template <class T>
__global__ void zero_pole_rows_kernel(cplx<T>* __restrict__ Y, int p, int Q) {
    const int b = blockIdx.x;
    cplx<T>* rowN = Y + (int64_t)b * Q * (p + 1);
    cplx<T>* rowS = rowN + (int64_t)(Q - 1) * (p + 1);
    for (int m = threadIdx.x; m <= p; m += blockDim.x) {
        rowN[m] = mk<T>(T(0), T(0));
        rowS[m] = mk<T>(T(0), T(0));
    }
}

// y <- x - y (n reals)
template <class T>
__global__ void residual_kernel(const T* __restrict__ x, T* __restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[i] - y[i];
}

// y <- y + x (n reals)
template <class T>
__global__ void accumulate_kernel(const T* __restrict__ x, T* __restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += x[i];
}

template <class T>
void launch_sh_adjoint(const hpx_plan_s* P, const T* maps, T* alm, cudaStream_t s, T scale) {
    const auto& g = P->g;
    launch_ring_fft<T>(P, maps, s, scale);
    zero_pole_rows_kernel<T><<<g.B, 256, 0, s>>>((cplx<T>*)P->Y, g.p, g.Q);
    launch_spread<T>(P, s);
    launch_lat_fft<T>(P, s);
    if (P->synM) {
        launch_fused<T>(P, alm, s, P->synM);
    } else {
        launch_dense<T>(P, s, P->t.Es);
        launch_rot<T>(P, alm, s);
    }
}

template <class T>
void launch_healpix_jacobi(const hpx_plan_s* P, const T* maps, T* alm, int niter, cudaStream_t s) {
    const auto& g = P->g;
    const T w = T(4.0 * 3.14159265358979323846 / (double)g.npix);   // 4 pi / N
    const int64_t nmap = g.B * g.npix, nalm = g.B * g.nalm * 2;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8;
    launch_sh_adjoint<T>(P, maps, alm, s, w);   // a = A f
    for (int k = 0; k < niter; ++k) {
        launch_sh_synthesis<T>(P, alm, (T*)P->jres, s);                           // S a
        residual_kernel<T><<<blocks, 256, 0, s>>>(maps, (T*)P->jres, nmap);        // r = f - S a
        launch_sh_adjoint<T>(P, (const T*)P->jres, (T*)P->jalm, s, w);           // A r
        accumulate_kernel<T><<<blocks, 256, 0, s>>>((const T*)P->jalm, alm, nalm);   // a += A r
    }
}

template void launch_sh_adjoint<float>(const hpx_plan_s*, const float*, float*, cudaStream_t, float);
template void launch_sh_adjoint<double>(const hpx_plan_s*, const double*, double*, cudaStream_t, double);
template void launch_healpix_jacobi<float>(const hpx_plan_s*, const float*, float*, int, cudaStream_t);
template void launch_healpix_jacobi<double>(const hpx_plan_s*, const double*, double*, int, cudaStream_t);

}  // namespace hpx
