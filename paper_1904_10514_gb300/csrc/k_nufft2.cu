// Type-2 direction of the latitude NUFFT (Sec. 3.2.2): from the latitude
// Fourier coefficients of every column (m, map) to values at the 4 Nside + 1
// latitude nodes.  It is the exact transpose of the analysis NUFFT of
// k_nufft.cu (deconvolution, M-point FFT, half-grid spreading with folded
// mirrors), used by hpx_synthesize and, with the synthesis coefficients as
// input, by hpx_sh_synthesis.  The inputs and outputs are those of
// nufft_adj_kernel (k_adjoint.cu):
//     even m:  y_r = w_r sum_j X_j cos(j theta_r)   (w_r = 2 on rings, 1 at poles)
//     odd m:   y_r = sum_j X_j sin(j theta_r)
// with X_j = bvec[b][m][j & 1][j >> 1] (odd m: the conj(i/2)-scaled sine
// coefficients of the analysis' right-hand-side convention).
//
// Two kernels, the transposes of lat_fft_pair and spread_rb:
//   ifft_pair_ct_kernel  one block per pair of orders (m even, m + 1) and map:
//       the transposed truncation puts the deconvolved coefficients c_j on j = 0..p;
//       the transposed symmetric extension of the half grid folds them into the
//       two-sided spectra U_j = c_j, U_{-j} = s c_j, U_0 = (1 + s) c_0 (s = +1 for
//       even m, -1 for odd m), so the half grid is v(t) = IFFT(U)(t) for
//       0 < t < M/2 and half of it at t = 0 and t = M/2.  The even order's grid
//       is symmetric and the odd order's antisymmetric, so one inverse FFT of
//       the sum of the two spectra gives both: v_m = (z(t) + z(M - t))/2,
//       v_{m+1} = (z(t) - z(M - t))/2.  Output: U[b][m][t], t = 0..M/2.
//   interp_rb_kernel  the transpose of the half-grid spreading: node r takes the
//       grid points tstart[r] .. tstart[r] + E - 1 with the spreading weights of
//       (grid point, node) (table hwn, one per parity of m).  A block takes 32
//       nodes of one map and loops over all orders 32 at a time (lane = order,
//       warp = 4 nodes, weights in registers), staging each order tile's grid
//       window through shared memory, and writes 32 contiguous orders per node
//       row of Y.
#include "fft_ct.cuh"
#include "plan.h"

namespace hpx {

template <int LOGM, int NT>
__global__ void __launch_bounds__(NT, (LOGM <= 13 ? 1024 / NT : 1)) ifft_pair_ct_kernel(
    const cplx<float>* __restrict__ bvec, cplx<float>* __restrict__ U, const float* __restrict__ dec,
    const cplx<float>* __restrict__ tw, int twlen, int p, int L, int P2, int ldu) {
    constexpr int M = 1 << LOGM;
    constexpr int H = M >> 1;
    extern __shared__ unsigned char smem_raw[];
    cplx<float>* buf = reinterpret_cast<cplx<float>*>(smem_raw);   // M (padded)
    const int m0 = 2 * blockIdx.x, m1 = m0 + 1;
    const int b = blockIdx.y;
    const int tid = threadIdx.x;
    const bool has1 = m1 <= L;
    const cplx<float>* in0 = bvec + ((int64_t)b * (p + 1) + m0) * 2 * P2;
    const cplx<float>* in1 = in0 + 2 * P2;
    auto c0 = [&](int j) { return scale(in0[(j & 1) * P2 + (j >> 1)], dec[j]); };
    auto c1 = [&](int j) {
        if (!has1) return mk<float>(0.f, 0.f);
        const cplx<float> v = in1[(j & 1) * P2 + (j >> 1)];
        return scale(mk<float>(0.5f * v.i, -0.5f * v.r), dec[j]);   // conj(i/2) v
    };
    auto ld = [&](int j, int) {
        if (j == 0) return scale(c0(0), 2.f);
        if (j <= p) return add(c0(j), c1(j));
        if (j >= M - p) return sub(c0(M - j), c1(M - j));
        return mk<float>(0.f, 0.f);
    };
    ct::fft<float, LOGM, NT, true, false>(buf, tw, twlen >> LOGM, ld,
                                          [&](int, int pi, cplx<float> v) { buf[pi] = v; });
    cplx<float>* out0 = U + ((int64_t)b * (L + 1) + m0) * ldu;
    cplx<float>* out1 = out0 + ldu;
    for (int t = tid; t <= H; t += NT) {
        const cplx<float> z = buf[ct::padc(t)], zr = buf[ct::padc((M - t) & (M - 1))];
        cplx<float> v0 = scale(add(z, zr), 0.5f);
        if (t == 0 || t == H) v0 = scale(v0, 0.5f);
        out0[t] = v0;
        if (has1) out1[t] = scale(sub(z, zr), 0.5f);
    }
}

__device__ __forceinline__ void cp_async_commit2() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// EW: taps per node at most, DM: spread of tstart over 4 consecutive nodes at
// most, NS: order tiles in flight.  nrw: grid points per staged row (rounded
// up to an odd stride against bank conflicts).
template <int EW, int DM, int NS>
__global__ void __launch_bounds__(256, 2) interp_rb_kernel(const cplx<float>* __restrict__ U,
                                                           cplx<float>* __restrict__ Y,
                                                           const int* __restrict__ tstart,
                                                           const float* __restrict__ hwn, int E, int H, int p,
                                                           int Q, int L, int ldu, int nrw) {
    constexpr int W = EW + DM;
    extern __shared__ unsigned char smem_raw[];
    cplx<float>* out = reinterpret_cast<cplx<float>*>(smem_raw);   // [32 nodes][33]
    cplx<float>* us0 = out + 32 * 33;                              // NS x [32 orders][nrw]
    const int r0 = blockIdx.x * 32, b = blockIdx.y;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int T0 = tstart[r0];
    const int rf = min(r0 + 4 * warp, Q - 1);
    const int base = tstart[rf] - T0;   // window start of this warp's nodes, relative to T0
    const int par = lane & 1;           // order tiles start at multiples of 32
    float w[4][W];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int r = r0 + 4 * warp + j;
        const int off = (r < Q) ? tstart[r] - tstart[rf] : 0;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const int e = q - off;
            w[j][q] = (r < Q && e >= 0 && e < E) ? hwn[((size_t)e * Q + r) * 2 + par] : 0.f;
        }
    }
    const cplx<float>* ub = U + (int64_t)b * (L + 1) * ldu;
    auto fetch = [&](int m0, cplx<float>* us) {
        for (int idx = tid; idx < 32 * nrw; idx += 256) {
            const int ml = idx / nrw, tt = idx - ml * nrw;
            const int m = m0 + ml, t = T0 + tt;
            const bool ok = m <= L && t <= H;
            cp_async8(us + idx, ok ? ub + (int64_t)m * ldu + t : ub, ok ? 8 : 0);
        }
        cp_async_commit2();
    };
    const int ntiles = (L + 32) / 32;
#pragma unroll
    for (int q = 0; q < NS - 1; ++q) {
        if (q < ntiles) fetch(32 * q, us0 + q * 32 * nrw);
        else cp_async_commit2();
    }
    for (int it = 0; it < ntiles; ++it) {
        const int m0 = 32 * it;
        cplx<float>* us = us0 + (it % NS) * 32 * nrw;
        if (it + NS - 1 < ntiles) fetch(m0 + 32 * (NS - 1), us0 + ((it + NS - 1) % NS) * 32 * nrw);
        else cp_async_commit2();
        cp_async_wait2<NS - 1>();
        __syncthreads();
        float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};
        const cplx<float>* ur = us + lane * nrw + base;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const cplx<float> v = ur[q];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                ar[j] += w[j][q] * v.r;
                ai[j] += w[j][q] * v.i;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) out[(4 * warp + j) * 33 + lane] = mk<float>(ar[j], ai[j]);
        __syncthreads();
        for (int idx = tid; idx < 32 * 32; idx += 256) {
            const int rl = idx >> 5, ml = idx & 31;
            const int r = r0 + rl, m = m0 + ml;
            if (r < Q && m <= L) Y[((int64_t)b * Q + r) * (p + 1) + m] = out[rl * 33 + ml];
        }
    }
}

// Returns false where these kernels do not apply (FP64 plans, grids outside
// 4096..16384 points, wider interpolation runs); the caller then runs
// nufft_adj_kernel.
bool launch_nufft2(const hpx_plan_s* P, cudaStream_t s) {
    const auto& g = P->g;
    const auto& t = P->t;
    constexpr int EW = 12, DM = 4, NS = 3;
    if (P->precision != HPX_FP32 || !t.tstart || t.interpE > EW || t.interpD > DM) return false;
    int logM = 0;
    while ((1 << logM) < g.M) ++logM;
    if (logM < 12 || logM > 14) return false;
    const size_t smem1 = (size_t)(g.M + g.M / 16) * sizeof(cplx<float>);
    dim3 grid1((g.L + 2) / 2, g.B);
    auto run1 = [&](auto kern, int threads) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
        kern<<<grid1, threads, smem1, s>>>((const cplx<float>*)P->bvec, (cplx<float>*)P->U, (const float*)t.dec,
                                           (const cplx<float>*)t.twid, g.Lmax, g.p, g.L, g.P2, P->ldu);
    };
    if (logM == 12) run1(ifft_pair_ct_kernel<12, 256>, 256);
    else if (logM == 13) run1(ifft_pair_ct_kernel<13, 512>, 512);
    else run1(ifft_pair_ct_kernel<14, 512>, 512);
    const int nrw = (t.interpRows + EW + DM) | 1;
    const size_t smem2 = (size_t)(32 * 33 + NS * 32 * nrw) * sizeof(cplx<float>);
    auto kern2 = interp_rb_kernel<EW, DM, NS>;
    cudaFuncSetAttribute(kern2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    dim3 grid2((g.Q + 31) / 32, g.B);
    kern2<<<grid2, 256, smem2, s>>>((const cplx<float>*)P->U, (cplx<float>*)P->Y, t.tstart, (const float*)t.hwn,
                                    t.interpE, g.M / 2, g.p, g.Q, g.L, P->ldu, nrw);
    return true;
}

}  // namespace hpx
