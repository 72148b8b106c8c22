// Latitude least-squares solve and change of basis to order-0/1 normalised
// Legendre functions (Sec. 3.2.2 and the first half of Sec. 3.3).
//
// For every column (map, m) the LS solution of the truncated normal equations
// T g = b (T = F^* F restricted to the m = 4 Nside + 1 latitude modes, split by
// the DFS parity of m into a cosine and a sine system) is followed by the
// projection of the resulting latitude series onto Pbar_l^0 (m even) or Pbar_l^1
// (m odd), scaled by sqrt(2 pi).  Both maps are fixed and shared by all columns
// and maps, so the plan premultiplies them (FP64) into one dense operator per
// (parity of m, parity of l):  beta = D b.  This kernel is that multi-column
// contraction:  beta[m][par][q][b][re/im] = sum_k D[m&1][par][q][k] * bvec[b][m][par][k].
// The output is column-contiguous (all maps of one (m, par, q) side by side) for
// the rotation sweeps, which process one real column per lane.
#include "plan.h"

namespace hpx {

namespace {
constexpr int TQ = 64;   // rows (q) per block
constexpr int TC = 32;   // columns (map, m) per block
constexpr int TK = 16;   // k per stage
}  // namespace

template <class T>
__global__ void __launch_bounds__(256) dense_kernel(const T* __restrict__ D,
                                                    const cplx<T>* __restrict__ bvec,
                                                    cplx<T>* __restrict__ beta, int P2, int p, int L,
                                                    int B) {
    __shared__ T Ds[TK][TQ + 1];
    __shared__ cplx<T> Bs[TK][TC + 1];   // padded: the loads below store 16 consecutive k of one column
    const int mpar = blockIdx.z >> 1, par = blockIdx.z & 1;
    const int nmp = (L >= mpar) ? (L - mpar) / 2 + 1 : 0;
    const int ncols = nmp * B;
    const int c0 = blockIdx.x * TC, q0 = blockIdx.y * TQ;
    if (c0 >= ncols) return;
    const T* Dm = D + ((size_t)(mpar * 2 + par) * P2) * P2;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;   // 4 rows x 2 columns per thread
    T accr[4][2], acci[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 2; ++c) { accr[a][c] = T(0); acci[a][c] = T(0); }

    for (int k0 = 0; k0 < P2; k0 += TK) {
        for (int e = tid; e < TQ * TK; e += 256) {
            const int qq = e / TK, kk = e % TK;
            const int q = q0 + qq, k = k0 + kk;
            Ds[kk][qq] = (q < P2 && k < P2) ? Dm[(size_t)q * P2 + k] : T(0);
        }
        for (int e = tid; e < TC * TK; e += 256) {
            const int cc = e / TK, kk = e % TK;
            const int col = c0 + cc, k = k0 + kk;
            cplx<T> v = mk<T>(T(0), T(0));
            if (col < ncols && k < P2) {
                const int b = col % B, mi = col / B;
                const int m = 2 * mi + mpar;
                v = bvec[(((int64_t)b * (p + 1) + m) * 2 + par) * P2 + k];
            }
            Bs[kk][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            T a[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = Ds[kk][tx * 4 + r];
            cplx<T> bb[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) bb[c] = Bs[kk][ty * 2 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    accr[r][c] += a[r] * bb[c].r;
                    acci[r][c] += a[r] * bb[c].i;
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int col = c0 + ty * 2 + c;
        if (col >= ncols) continue;
        const int b = col % B, mi = col / B;
        const int m = 2 * mi + mpar;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int q = q0 + tx * 4 + r;
            if (q < P2) beta[(((int64_t)m * 2 + par) * P2 + q) * B + b] = mk<T>(accr[r][c], acci[r][c]);
        }
    }
}

template <class T>
void launch_dense(const hpx_plan_s* P, cudaStream_t s, const void* Dmat) {
    const auto& g = P->g;
    const int nmp = g.L / 2 + 1;
    dim3 grid((nmp * g.B + TC - 1) / TC, (g.P2 + TQ - 1) / TQ, 4);
    dense_kernel<T><<<grid, 256, 0, s>>>((const T*)(Dmat ? Dmat : P->t.D), (const cplx<T>*)P->bvec, (cplx<T>*)P->beta,
                                         g.P2, g.p, g.L, g.B);
}

template void launch_dense<float>(const hpx_plan_s*, cudaStream_t, const void*);
template void launch_dense<double>(const hpx_plan_s*, cudaStream_t, const void*);

}  // namespace hpx
