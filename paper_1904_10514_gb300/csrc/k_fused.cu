// Per-order operators: the latitude least-squares solve, the change of basis to
// order-0/1 Legendre functions (operator D) and the m/2 Givens sweeps of
// Sec. 3.3 are all fixed linear maps, so for every order m and parity chain c
// their composition is one matrix
//     M_{m,c} = R_{m,c} D_par[rows of chain c],   N(m,c) x P2,
// with R_{m,c} the product of the sweeps.  The plan builds every M_{m,c} once,
// in FP64 on the GPU, by running the same register-wavefront sweeps over the
// columns of D (build_fused_kernel), and stores it rounded to the plan precision
// (n_alm x P2 entries in total, 8.6 GB in FP32 at lmax 2048).  The analysis then
// needs one multi-map contraction per (m, c) instead of the dense stage and the
// run-time sweeps (fused_apply_kernel):
//     a_{m+c+2i}^m[map] = sum_k M_{m,c}[i][k] * b[map][m][par][k].
#include <algorithm>

#include "plan.h"
#include "plan_math.h"
#include "sweep.cuh"

namespace hpx {

// ---------------------------------------------------------------- build (FP64)
// One warp per (m, chain c, group of 32 complex columns); complex column j holds
// the real columns 2j and 2j+1 of D.  The chain of each lane lives in `scratch`.
template <class T>
__global__ void __launch_bounds__(64) build_fused_kernel(const double* __restrict__ D, T* __restrict__ Mout,
                                                         const int64_t* __restrict__ moff,
                                                         const int64_t* __restrict__ skOff,
                                                         const cplx<double>* __restrict__ skew, int nq, int P2,
                                                         int ldm, int L, int m_lo, int m_cnt, int ngroups,
                                                         cplx<double>* __restrict__ scratch,
                                                         const int64_t* __restrict__ tcOff,
                                                         const int* __restrict__ tcFirst) {
    constexpr int KMAX = 16;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nitems = m_cnt * 2 * ngroups;
    if (warp >= nitems) return;
    const int g = warp % ngroups;
    const int c = (warp / ngroups) & 1;
    const int mi = warp / (2 * ngroups);
    const int m = m_lo + mi;
    const int m0 = m & 1;
    const int S = (m - m0) >> 1;
    const int ncplx = (P2 + 1) / 2;
    const int j = 32 * g + lane;
    if (j >= ncplx) return;
    const int par = (m0 + c) & 1;
    const int q0 = (m0 == 1 && c == 1) ? 1 : 0;
    cplx<double>* chain = scratch + ((int64_t)mi * 2 + c) * P2 * ncplx + j;
    const int64_t ldc = ncplx;
    const double* Dp = D + ((size_t)(m0 * 2 + par) * P2) * P2;
    int n = chain_len(m0, c, L);
    for (int i = 0; i < n; ++i) {
        const double* row = Dp + (size_t)(q0 + i) * P2;
        chain[(int64_t)i * ldc] = mk<double>(row[2 * j], (2 * j + 1 < P2) ? row[2 * j + 1] : 0.0);
    }
    int s0 = 0;
    auto block = [&](int s) {
        return skew + (skOff[(size_t)(m0 * 2 + c) * nq + (s >> 5)] + 2 * (s & 31)) * 32;
    };
    while (S - s0 >= KMAX && n > 0) {
        sweep_pass<double, KMAX>(chain, ldc, n, block(s0), s0 & 31);
        n -= KMAX;
        s0 += KMAX;
    }
#define HPX_SUBPASS(KK)                                                   \
    if (S - s0 >= KK && n > 0) {                                          \
        sweep_pass<double, KK>(chain, ldc, n, block(s0), s0 & 31);        \
        n -= KK;                                                          \
        s0 += KK;                                                         \
    }
    HPX_SUBPASS(8)
    HPX_SUBPASS(4)
    HPX_SUBPASS(2)
    HPX_SUBPASS(1)
#undef HPX_SUBPASS
    if (tcOff) {   // tensor-core layout (FP32 plans)
        for (int i = 0; i < n; ++i) {
            const cplx<double> v = chain[(int64_t)i * ldc];
            const int rp = (min(128, n - (i & ~127)) + 7) & ~7;
            T* out = Mout + tcOff[tcFirst[m * 2 + c] + (i >> 7)];
            out[tc_elem(rp, i & 127, 2 * j)] = (T)v.r;
            if (2 * j + 1 < P2) out[tc_elem(rp, i & 127, 2 * j + 1)] = (T)v.i;
        }
        return;
    }
    T* out = Mout + moff[(size_t)m * 2 + c] * ldm;
    for (int i = 0; i < n; ++i) {
        const cplx<double> v = chain[(int64_t)i * ldc];
        out[(size_t)i * ldm + 2 * j] = (T)v.r;
        if (2 * j + 1 < P2) out[(size_t)i * ldm + 2 * j + 1] = (T)v.i;
    }
}

// ---------------------------------------------------------------- apply

// Block = one (m, c, tile of 8*TR rows) x 2*TC maps; TR*TC threads, each 8 rows x 2 maps.
// M rows are padded to ldm (a multiple of 4, zero filled) so that they load as
// 16-byte vectors.
template <class T, int TR, int TC>
__global__ void __launch_bounds__(TR* TC) fused_apply_kernel(const T* __restrict__ M, const int64_t* __restrict__ moff,
                                                             const int* __restrict__ tiles,
                                                             const cplx<T>* __restrict__ bvec,
                                                             cplx<T>* __restrict__ alm, int P2, int ldm, int p,
                                                             int L, int B, int64_t nalm) {
    constexpr int FR = 8 * TR, FC = 2 * TC, NT = TR * TC;
    constexpr int FK = sizeof(T) == 4 ? 16 : 8;   // k per stage
    constexpr int VA = 16 / sizeof(T);            // elements per 16-byte vector
    __shared__ __align__(16) T As[FK][FR + 4];
    __shared__ __align__(16) cplx<T> Bs[FK][FC];
    const int m = tiles[3 * blockIdx.x], c = tiles[3 * blockIdx.x + 1], i0 = tiles[3 * blockIdx.x + 2];
    const int m0 = m & 1;
    const int par = (m0 + c) & 1;
    const int nrows = chain_len(m, c, L);
    const int b0 = blockIdx.y * FC;
    const T* A = M + moff[(size_t)m * 2 + c] * ldm;
    const int tid = threadIdx.x;
    const int tr = tid % TR, tc = tid / TR;
    T accr[8][2], acci[8][2];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 2; ++q) { accr[r][q] = T(0); acci[r][q] = T(0); }

    for (int k0 = 0; k0 < P2; k0 += FK) {
        // A tile: FR rows x 16 k as 16-byte vectors, stored k-major
        for (int e = tid; e < FR * (FK / VA); e += NT) {
            const int rr = e % FR, kv = e / FR;   // a warp stores 32 consecutive rows: no bank conflicts
            const int i = i0 + rr, k = k0 + kv * VA;
            T v[VA];
            if (i < nrows && k < ldm) {
                if constexpr (sizeof(T) == 4) {
                    const float4 q4 = *reinterpret_cast<const float4*>(A + (size_t)i * ldm + k);
                    v[0] = q4.x; v[1] = q4.y; v[2] = q4.z; v[3] = q4.w;
                } else {
                    const double2 q2 = *reinterpret_cast<const double2*>(A + (size_t)i * ldm + k);
                    v[0] = q2.x; v[1] = q2.y;
                }
            } else {
#pragma unroll
                for (int q = 0; q < VA; ++q) v[q] = T(0);
            }
#pragma unroll
            for (int q = 0; q < VA; ++q) As[kv * VA + q][rr] = v[q];
        }
        // B tile: FC maps x 16 k (each map's column is contiguous in k)
        for (int e = tid; e < FC * FK; e += NT) {
            const int cc = e / FK, kk = e % FK;
            const int b = b0 + cc, k = k0 + kk;
            Bs[kk][cc] = (b < B && k < P2) ? bvec[(((int64_t)b * (p + 1) + m) * 2 + par) * P2 + k]
                                           : mk<T>(T(0), T(0));
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < FK; ++kk) {
            T a[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) a[r] = As[kk][tr * 8 + r];
            const cplx<T> x0 = Bs[kk][tc * 2], x1 = Bs[kk][tc * 2 + 1];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                accr[r][0] += a[r] * x0.r;
                acci[r][0] += a[r] * x0.i;
                accr[r][1] += a[r] * x1.r;
                acci[r][1] += a[r] * x1.i;
            }
        }
        __syncthreads();
    }
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2 + m + c;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int b = b0 + tc * 2 + q;
        if (b >= B) continue;
        cplx<T>* out = alm + (int64_t)b * nalm + base;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int i = i0 + tr * 8 + r;
            if (i < nrows) out[2 * i] = mk<T>(accr[r][q], acci[r][q]);
        }
    }
}

// ---------------------------------------------------------------- synthesis apply
// The synthesis direction of the same composition: with Es the Legendre-0/1 ->
// latitude-Fourier table in place of D, the build gives S_{m,c} = R_{m,c} Es
// (rows i = degrees of the chain, columns k = latitude modes), and the
// cosine/sine coefficients of F_m are the transposed contraction
//     X[map][m][par][k] = sum_i S_{m,c}[i][k] a_{m+c+2i}^m[map].
// Block = one (m, c, tile of 128 modes) x MB maps (16, or 32 so that batches of
// 17+ maps read each operator once); 256 threads, each 4 modes x MB/8 maps;
// degrees in chunks of 16 staged in shared memory.
template <class T, int MB>
__global__ void __launch_bounds__(256) synth_apply_kernel(const T* __restrict__ S, const int64_t* __restrict__ moff,
                                                          const cplx<T>* __restrict__ alm, cplx<T>* __restrict__ bvec,
                                                          int P2, int ldm, int p, int L, int B, int64_t nalm,
                                                          int nkt) {
    constexpr int KT = 128, IC = 16, QB = MB / 8;
    __shared__ __align__(16) T As[IC][KT];
    __shared__ cplx<T> Bs[IC][MB];
    const int item = blockIdx.x;
    const int kt = item % nkt, mc = item / nkt;
    const int m = mc >> 1, c = mc & 1;
    const int par = ((m & 1) + c) & 1;
    const int nrows = chain_len(m, c, L);
    const int k0 = kt * KT, b0 = blockIdx.y * MB;
    const T* A = S + moff[(size_t)m * 2 + c] * ldm;
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2 + m + c;
    const int tid = threadIdx.x, tk = tid & 31, tb = tid >> 5;
    T accr[4][QB], acci[4][QB];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < QB; ++q) { accr[a][q] = T(0); acci[a][q] = T(0); }
    for (int i0 = 0; i0 < nrows; i0 += IC) {
        for (int e = tid; e < IC * KT; e += 256) {
            const int ii = e / KT, kk = e % KT;
            const int i = i0 + ii, k = k0 + kk;
            As[ii][kk] = (i < nrows && k < ldm) ? A[(size_t)i * ldm + k] : T(0);
        }
        for (int e = tid; e < IC * MB; e += 256) {
            const int ii = e / MB, bb = e % MB;
            const int i = i0 + ii, b = b0 + bb;
            Bs[ii][bb] = (i < nrows && b < B) ? alm[(int64_t)b * nalm + base + 2 * i] : mk<T>(T(0), T(0));
        }
        __syncthreads();
#pragma unroll
        for (int ii = 0; ii < IC; ++ii) {
            T a[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[ii][tk * 4 + r];
            cplx<T> x[QB];
#pragma unroll
            for (int q = 0; q < QB; ++q) x[q] = Bs[ii][tb * QB + q];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < QB; ++q) {
                    accr[r][q] += a[r] * x[q].r;
                    acci[r][q] += a[r] * x[q].i;
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < QB; ++q) {
        const int b = b0 + tb * QB + q;
        if (b >= B) continue;
        cplx<T>* out = bvec + (((int64_t)b * (p + 1) + m) * 2 + par) * P2;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int k = k0 + tk * 4 + r;
            if (k < P2) out[k] = mk<T>(accr[r][q], acci[r][q]);
        }
    }
}

template <class T>
void launch_synth_apply(const hpx_plan_s* P, const T* alm, cudaStream_t s) {
    const auto& g = P->g;
    const int nkt = (g.P2 + 127) / 128;
    if (g.B > 16) {
        dim3 grid((g.L + 1) * 2 * nkt, (g.B + 31) / 32);
        synth_apply_kernel<T, 32><<<grid, 256, 0, s>>>((const T*)P->synM, P->fusedOff, (const cplx<T>*)alm,
                                                       (cplx<T>*)P->bvec, g.P2, P->fused_ldm, g.p, g.L, g.B, g.nalm,
                                                       nkt);
    } else {
        dim3 grid((g.L + 1) * 2 * nkt, (g.B + 15) / 16);
        synth_apply_kernel<T, 16><<<grid, 256, 0, s>>>((const T*)P->synM, P->fusedOff, (const cplx<T>*)alm,
                                                       (cplx<T>*)P->bvec, g.P2, P->fused_ldm, g.p, g.L, g.B, g.nalm,
                                                       nkt);
    }
}

template void launch_synth_apply<float>(const hpx_plan_s*, const float*, cudaStream_t);
template void launch_synth_apply<double>(const hpx_plan_s*, const double*, cudaStream_t);

// Rows per block of the apply kernel for a batch of B maps (the plan builds its
// tile list with this).
int fused_tile_rows(int B) { return B > 8 ? 128 : (B > 2 ? 256 : 512); }

template <class T>
void launch_fused(const hpx_plan_s* P, T* alm, cudaStream_t s, const void* Mrows) {
    const auto& g = P->g;
    const int ldm = P->fused_ldm;
    const T* M = (const T*)(Mrows ? Mrows : P->fusedM);
    if (g.B > 8) {
        dim3 grid(P->fused_ntiles, (g.B + 31) / 32);
        fused_apply_kernel<T, 16, 16><<<grid, 256, 0, s>>>(M, P->fusedOff, P->fusedTiles,
                                                           (const cplx<T>*)P->bvec, (cplx<T>*)alm, g.P2, ldm,
                                                           g.p, g.L, g.B, g.nalm);
    } else if (g.B > 2) {
        dim3 grid(P->fused_ntiles, (g.B + 7) / 8);
        fused_apply_kernel<T, 32, 4><<<grid, 128, 0, s>>>(M, P->fusedOff, P->fusedTiles,
                                                          (const cplx<T>*)P->bvec, (cplx<T>*)alm, g.P2, ldm,
                                                          g.p, g.L, g.B, g.nalm);
    } else {
        dim3 grid(P->fused_ntiles, (g.B + 1) / 2);
        fused_apply_kernel<T, 64, 1><<<grid, 64, 0, s>>>(M, P->fusedOff, P->fusedTiles,
                                                         (const cplx<T>*)P->bvec, (cplx<T>*)alm, g.P2, ldm,
                                                         g.p, g.L, g.B, g.nalm);
    }
}

// Builds the per-order operators of a plan (called once by hpx_plan_ex).
// D64 / skew64 are FP64 device copies of D and of the skewed sweep angles.
template <class T>
int build_fused(hpx_plan_s* P, const double* D64, const cplx<double>* skew64, cudaStream_t s, void* out,
                bool tiled) {
    const auto& g = P->g;
    const int ncplx = (g.P2 + 1) / 2;
    const int ngroups = (ncplx + 31) / 32;
    const int chunk = 64;
    cplx<double>* scratch = nullptr;
    const size_t sbytes = (size_t)chunk * 2 * g.P2 * ncplx * sizeof(cplx<double>);
    if (cudaMalloc(&scratch, sbytes) != cudaSuccess) return -1;
    for (int m_lo = 0; m_lo <= g.L; m_lo += chunk) {
        const int m_cnt = std::min(chunk, g.L + 1 - m_lo);
        const int nitems = m_cnt * 2 * ngroups;
        const int blocks = (nitems * 32 + 63) / 64;
        build_fused_kernel<T><<<blocks, 64, 0, s>>>(D64, (T*)out, P->fusedOff, P->t.skOff, skew64, P->t.nq,
                                                    g.P2, P->fused_ldm, g.L, m_lo, m_cnt, ngroups, scratch,
                                                    tiled ? P->tcOff : nullptr, P->tcFirst);
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(scratch);
    return e == cudaSuccess ? 0 : -1;
}

template void launch_fused<float>(const hpx_plan_s*, float*, cudaStream_t, const void*);
template void launch_fused<double>(const hpx_plan_s*, double*, cudaStream_t, const void*);
template int build_fused<float>(hpx_plan_s*, const double*, const cplx<double>*, cudaStream_t, void*, bool);
template int build_fused<double>(hpx_plan_s*, const double*, const cplx<double>*, cudaStream_t, void*, bool);

}  // namespace hpx
