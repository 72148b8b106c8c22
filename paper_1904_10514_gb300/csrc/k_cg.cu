// Conjugate-gradient form of the latitude least squares (Sec. 3.2.2):
// instead of applying the premultiplied inverse, each column's normal equations
//     T g = b     (T = the Toeplitz-plus-Hankel Gram matrix of the cosine or
//                  sine basis at the latitude nodes, one per parity of m and j)
// are solved by CG, with T x = IFFT(Hc . FFT(x) + Hg . FFT(x)(-k)) restricted to
// the first n entries (one forward and one inverse N-point FFT in shared memory
// per iteration; tables from build_cg_tables).  The solution overwrites the
// right-hand side in bvec; the change of basis to order-0/1 Legendre
// coefficients (C) and the Givens sweeps follow as in the sweeps path.
#include "plan.h"

namespace hpx {

namespace {
// block-wide sum of one double per thread (blockDim a multiple of 32, <= 1024)
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    return s;
}
}  // namespace

template <class T, int E>
__global__ void __launch_bounds__(512, 1) cg_kernel(cplx<T>* __restrict__ bvec, const cplx<T>* __restrict__ H,
                                                 int4 k0s, int4 ns, int N, int logN,
                                                 const cplx<T>* __restrict__ tw, int twlen, int p, int P2,
                                                 double tol2, int maxit) {
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);   // N (padded)
    const int nmax = max(max(ns.x, ns.y), max(ns.z, ns.w));
    cplx<T>* x = buf + N + N / 16;
    cplx<T>* r = x + nmax;
    cplx<T>* pv = r + nmax;
    cplx<T>* q = pv + nmax;
    __shared__ double red[32];
    const int m = blockIdx.x, b = blockIdx.y;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int mpar = m & 1;
    for (int par = 0; par < 2; ++par) {
        const int blk = 2 * mpar + par;
        const int k0 = blk == 0 ? k0s.x : blk == 1 ? k0s.y : blk == 2 ? k0s.z : k0s.w;
        const int n = blk == 0 ? ns.x : blk == 1 ? ns.y : blk == 2 ? ns.z : ns.w;
        if (n == 0) continue;
        cplx<T>* bb = bvec + (((int64_t)b * (p + 1) + m) * 2 + par) * P2 + k0;
        const cplx<T>* Hc = H + (size_t)blk * 2 * N;
        const cplx<T>* Hg = Hc + N;
        double rr = 0.0;
        for (int i = tid; i < n; i += nt) {
            const cplx<T> v = bb[i];
            x[i] = mk<T>(T(0), T(0));
            r[i] = v;
            pv[i] = v;
            rr += (double)v.r * v.r + (double)v.i * v.i;
        }
        rr = block_sum(rr, red);
        const double stop = tol2 * rr;
        for (int it = 0; it < maxit && rr > stop; ++it) {
            // q = T pv
            for (int i = tid; i < N; i += nt) buf[pad(i)] = i < n ? pv[i] : mk<T>(T(0), T(0));
            __syncthreads();
            block_fft_pad<T, E>(buf, logN, tw, twlen, false);
            for (int k = tid; k <= N / 2; k += nt) {
                const int k2 = (N - k) & (N - 1);
                const cplx<T> X1 = buf[pad(k)], X2 = buf[pad(k2)];
                const cplx<T> Y1 = add(mul(Hc[k], X1), mul(Hg[k], X2));
                const cplx<T> Y2 = add(mul(Hc[k2], X2), mul(Hg[k2], X1));
                buf[pad(k)] = Y1;
                if (k2 != k) buf[pad(k2)] = Y2;
            }
            __syncthreads();
            block_fft_pad<T, E>(buf, logN, tw, twlen, true);
            double pq = 0.0;
            for (int i = tid; i < n; i += nt) {
                const cplx<T> v = buf[pad(i)];
                q[i] = v;
                pq += (double)pv[i].r * v.r + (double)pv[i].i * v.i;
            }
            pq = block_sum(pq, red);
            const T alpha = (T)(rr / pq);
            double rn = 0.0;
            for (int i = tid; i < n; i += nt) {
                x[i] = add(x[i], scale(pv[i], alpha));
                const cplx<T> v = sub(r[i], scale(q[i], alpha));
                r[i] = v;
                rn += (double)v.r * v.r + (double)v.i * v.i;
            }
            rn = block_sum(rn, red);
            const T beta = (T)(rn / rr);
            rr = rn;
            for (int i = tid; i < n; i += nt) pv[i] = add(r[i], scale(pv[i], beta));
            __syncthreads();
        }
        for (int i = tid; i < n; i += nt) bb[i] = x[i];
        __syncthreads();
    }
}

template <class T>
void launch_cg(const hpx_plan_s* P, cudaStream_t s) {
    const auto& g = P->g;
    const auto& t = P->t;
    int logN = 0;
    while ((1 << logN) < t.cgN) ++logN;
    int nmax = 0;
    for (int k = 0; k < 4; ++k) nmax = std::max(nmax, t.cgn[k]);
    const size_t smem = (size_t)(t.cgN + t.cgN / 16 + 4 * nmax) * sizeof(cplx<T>);
    auto kern = t.cgN > 16 * 512 ? cg_kernel<T, 32> : cg_kernel<T, 16>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const double tol = sizeof(T) == 4 ? 1e-7 : 1e-14;
    dim3 grid(g.L + 1, g.B);
    kern<<<grid, 512, smem, s>>>((cplx<T>*)P->bvec, (const cplx<T>*)t.cgH,
                                 make_int4(t.cgk0[0], t.cgk0[1], t.cgk0[2], t.cgk0[3]),
                                 make_int4(t.cgn[0], t.cgn[1], t.cgn[2], t.cgn[3]), t.cgN, logN,
                                 (const cplx<T>*)t.twid, g.Lmax, g.p, g.P2, tol * tol, sizeof(T) == 4 ? 60 : 120);
}

template void launch_cg<float>(const hpx_plan_s*, cudaStream_t);
template void launch_cg<double>(const hpx_plan_s*, cudaStream_t);

}  // namespace hpx
