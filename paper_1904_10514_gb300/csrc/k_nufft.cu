// Step 2 (Sec. 3.2): DFS doubling in latitude and the right-hand side of the
// least-squares inverse NUFFT-II, b = F^* y (the type-1 NUFFT of Sec. 3.2.2).
//
// For longitude wavenumber m the DFS data (remark of Sec. 3.2.1) are y_r at the
// latitudes theta_r (r = 0..4 Nside: poles and rings) and (-1)^m y_r at
// 2 pi - theta_r (interior r).  The type-1 sums
//     B_j = sum_nodes y_nu e^{-i j theta_nu},   j = 0..p,
// are computed with an exponential-of-semicircle (ES) kernel: the node values are
// spread onto a uniform grid of M = 8 Nside points on [0, 2 pi) (a gather over a
// precomputed sparse table, accumulated in shared memory), the grid is
// transformed by an M-point FFT in shared memory, and each mode is divided by
// the kernel's Fourier transform (table `dec`, FP64-built).
//
// By the DFS parity the LS problem splits (even m: cosine basis, odd m: sine
// basis); the outputs are the normal-equation right-hand sides
//     even m:  b_j = sum_r w_r y_r cos(j theta_r)          = B_j
//     odd m:   b_j = sum_{interior r} y_r sin(j theta_r)   = (i/2) B_j
// stored as bvec[b][m][j & 1][j >> 1].
#include "plan.h"

namespace hpx {

template <class T, int E>
__global__ void __launch_bounds__(512, (E <= 16 ? 2 : 1)) nufft_kernel(
    const cplx<T>* __restrict__ Y, cplx<T>* __restrict__ bvec, const int* __restrict__ nstart,
    const T* __restrict__ swts, int nsw, const T* __restrict__ dec, const cplx<T>* __restrict__ tw, int twlen, int M,
    int logM, int p, int Q, int P2) {
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* u = reinterpret_cast<cplx<T>*>(smem_raw);   // M
    cplx<T>* y = u + M + M / 16;                           // Q (after the padded grid)
    const int m = blockIdx.x;
    const int b = blockIdx.y;
    const int tid = threadIdx.x, nt = blockDim.x;
    const cplx<T>* col = Y + (int64_t)b * Q * (p + 1) + m;
    for (int r = tid; r < Q; r += nt) y[r] = col[(int64_t)r * (p + 1)];
    __syncthreads();
    const bool odd = (m & 1) != 0;
    // gather-spread: grid point t sees the DFS nodes nstart[t] .. nstart[t]+nsw-1
    // (cyclically; node nu <= 4 Nside is theta_nu, beyond it is the mirror of
    // ring 8 Nside - nu, whose data carry the sign (-1)^m); M = 8 Nside nodes.
    const int half = M >> 1;
    for (int t = tid; t < M; t += nt) {
        T ar = T(0), ai = T(0);
        int nu = nstart[t];
        for (int e = 0; e < nsw; ++e) {
            const T w = swts[(size_t)e * M + t];
            const bool mir = nu > half;
            const cplx<T> v = y[mir ? M - nu : nu];
            const T ws = (odd && mir) ? -w : w;
            ar += ws * v.r;
            ai += ws * v.i;
            nu = (nu + 1 == M) ? 0 : nu + 1;
        }
        u[pad(t)] = mk<T>(ar, ai);
    }
    __syncthreads();
    block_fft_pad<T, E>(u, logM, tw, twlen, false);
    cplx<T>* out = bvec + ((int64_t)b * (p + 1) + m) * 2 * P2;
    for (int j = tid; j <= p; j += nt) {
        cplx<T> v = scale(u[pad(j)], dec[j]);
        if (odd) v = mk<T>(T(-0.5) * v.i, T(0.5) * v.r);
        out[(j & 1) * P2 + (j >> 1)] = v;
    }
    // the odd-parity block has one slot fewer (j = p + 1 would be index p/2)
    if (tid == 0) out[P2 + (P2 - 1)] = mk<T>(T(0), T(0));
}

template <class T>
void launch_nufft(const hpx_plan_s* P, cudaStream_t s) {
    const auto& g = P->g;
    const auto& t = P->t;
    int logM = 0;
    while ((1 << logM) < g.M) ++logM;
    const size_t smem = (size_t)(g.M + g.M / 16 + g.Q) * sizeof(cplx<T>);
    auto kern = g.M > 16 * 512 ? nufft_kernel<T, 32> : nufft_kernel<T, 16>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid(g.L + 1, g.B);
    kern<<<grid, 512, smem, s>>>((const cplx<T>*)P->Y, (cplx<T>*)P->bvec, t.nstart, (const T*)t.swts, t.spreadE,
                                 (const T*)t.dec, (const cplx<T>*)t.twid, g.Lmax, g.M, logM, g.p, g.Q, g.P2);
}

template void launch_nufft<float>(const hpx_plan_s*, cudaStream_t);
template void launch_nufft<double>(const hpx_plan_s*, cudaStream_t);

}  // namespace hpx
