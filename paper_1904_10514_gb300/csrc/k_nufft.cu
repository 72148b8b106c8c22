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
//
// nufft_kernel does the whole step per column (used by the allocation-free
// entry point); plans run it as spread_kernel + lat_fft_kernel below.
#include "fft_ct.cuh"
#include "fp16pair.cuh"
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

// ---------------------------------------------------------------------------
// The same step as two kernels (the analysis path of plans):
//
// spread_kernel: the grid values obey u[M - t] = (-1)^m u[t], so only the half
// grid t = 0..M/2 is spread, with every mirrored node folded into its latitude
// node (weights hwts, one per parity of m).  A block takes 32 grid points x 32
// consecutive orders of one map: the ring coefficients of the latitude nodes it
// needs are read row by row (32 orders = 256 contiguous bytes), the 12 or so
// taps per grid point are summed from shared memory, and the 32 x 32 results
// are written transposed, as 32 contiguous half-grid segments of U[b][m][t].
template <class T>
__global__ void __launch_bounds__(256) spread_kernel(const cplx<T>* __restrict__ Y, cplx<T>* __restrict__ U,
                                                     const int* __restrict__ hstart, const T* __restrict__ hwts,
                                                     int E, int H, int p, int Q, int L, int ldu) {
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* out = reinterpret_cast<cplx<T>*>(smem_raw);   // [32 orders][33]
    cplx<T>* ys = out + 32 * 33;                           // [rows][32 orders]
    const int t0 = blockIdx.x * 32, m0 = blockIdx.y * 32, b = blockIdx.z;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R0 = hstart[t0];
    const int nr = hstart[min(t0 + 31, H)] + E - R0;
    const cplx<T>* yb = Y + (int64_t)b * Q * (p + 1);
    for (int idx = tid; idx < nr * 32; idx += 256) {
        const int r = idx >> 5, ml = idx & 31;
        const int m = m0 + ml;
        ys[idx] = (m <= L) ? yb[(int64_t)(R0 + r) * (p + 1) + m] : mk<T>(T(0), T(0));
    }
    __syncthreads();
    const int odd = (m0 + lane) & 1;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int tl = 4 * warp + j, t = t0 + tl;
        T ar = T(0), ai = T(0);
        if (t <= H) {
            const cplx<T>* yr = ys + (hstart[t] - R0) * 32 + lane;
            const T* w = hwts + 2 * t + odd;
            for (int e = 0; e < E; ++e) {
                const T we = w[(size_t)e * 2 * (H + 1)];
                const cplx<T> v = yr[32 * e];
                ar += we * v.r;
                ai += we * v.i;
            }
        }
        out[lane * 33 + tl] = mk<T>(ar, ai);
    }
    __syncthreads();
    for (int idx = tid; idx < 32 * 32; idx += 256) {
        const int ml = idx >> 5, tl = idx & 31;
        const int m = m0 + ml, t = t0 + tl;
        if (m <= L && t <= H) U[((int64_t)b * (L + 1) + m) * ldu + t] = out[ml * 33 + tl];
    }
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Register-blocked form for FP32 (at most EW taps, consecutive groups of 4 grid
// points starting at most DM latitude nodes apart): a block takes 32 grid points
// of one map and loops over all orders 32 at a time.  Warp w owns grid points
// t0 + 4w .. t0 + 4w + 3 and lane l order m0 + l; the thread keeps its 4 x EW
// weights (for the parity of its order) in registers, aligned to a common
// window of EW + DM latitude nodes, so every node value read from shared
// memory feeds four grid points.  The node values of the orders 32 .. 32 (NS-1)
// ahead are in flight (cp.async into a ring of NS buffers) while the current
// ones are used.
template <int EW, int DM, int NS>
__global__ void __launch_bounds__(256, 2) spread_rb_kernel(const cplx<float>* __restrict__ Y,
                                                           cplx<float>* __restrict__ U,
                                                           const int* __restrict__ hstart,
                                                           const float* __restrict__ hwts, int E, int H, int p,
                                                           int Q, int L, int ldu, int nrw) {
    constexpr int W = EW + DM;
    extern __shared__ unsigned char smem_raw[];
    cplx<float>* out = reinterpret_cast<cplx<float>*>(smem_raw);   // [32 orders][33]
    cplx<float>* ys0 = out + 32 * 33;                              // NS x [nrw rows][32 orders]
    const int t0 = blockIdx.x * 32, b = blockIdx.y;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R0 = hstart[t0];
    const int tf = min(t0 + 4 * warp, H);
    const int base = hstart[tf] - R0;   // window start, relative to R0
    const int par = lane & 1;           // m0 is a multiple of 32
    float w[4][W];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int t = t0 + 4 * warp + j;
        const int off = (t <= H) ? hstart[t] - hstart[tf] : 0;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const int e = q - off;
            w[j][q] = (t <= H && e >= 0 && e < E) ? hwts[((size_t)e * (H + 1) + t) * 2 + par] : 0.f;
        }
    }
    const cplx<float>* yb = Y + (int64_t)b * Q * (p + 1);
    auto fetch = [&](int m0, cplx<float>* ys) {
        for (int idx = tid; idx < nrw * 32; idx += 256) {
            const int r = idx >> 5, m = m0 + (idx & 31);
            const bool ok = m <= L && R0 + r < Q;
            cp_async8(ys + idx, ok ? yb + (int64_t)(R0 + r) * (p + 1) + m : yb, ok ? 8 : 0);
        }
        cp_async_commit();
    };
    const int ntiles = (L + 32) / 32;
    // one commit group per tile (empty past the last), so that waiting until at
    // most NS - 1 groups are pending means tile it has landed
#pragma unroll
    for (int q = 0; q < NS - 1; ++q) {
        if (q < ntiles) fetch(32 * q, ys0 + q * nrw * 32);
        else cp_async_commit();
    }
    for (int it = 0; it < ntiles; ++it) {
        const int m0 = 32 * it;
        cplx<float>* ys = ys0 + (it % NS) * nrw * 32;
        // buffer (it + NS - 1) % NS was last read in iteration it - 1, which
        // ended with a barrier
        if (it + NS - 1 < ntiles) fetch(m0 + 32 * (NS - 1), ys0 + ((it + NS - 1) % NS) * nrw * 32);
        else cp_async_commit();
        cp_async_wait<NS - 1>();
        __syncthreads();
        float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};
        const cplx<float>* yr = ys + base * 32 + lane;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const cplx<float> v = yr[32 * q];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                ar[j] += w[j][q] * v.r;
                ai[j] += w[j][q] * v.i;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) out[lane * 33 + 4 * warp + j] = mk<float>(ar[j], ai[j]);
        __syncthreads();
        for (int idx = tid; idx < 32 * 32; idx += 256) {
            const int ml = idx >> 5, tl = idx & 31;
            const int m = m0 + ml, t = t0 + tl;
            if (m <= L && t <= H) U[((int64_t)b * (L + 1) + m) * ldu + t] = out[ml * 33 + tl];
        }
    }
}

// lat_fft_kernel: one block per (order m, map): M-point FFT of the grid whose
// first pass reads the half grid from U (mirrored past M/2) and whose last pass
// deconvolves and writes the modes j <= p as the normal-equation right-hand
// sides (same output as nufft_kernel); the passes between run in shared memory.
template <class T, int E>
__global__ void __launch_bounds__(512, (E <= 16 ? 2 : 1)) lat_fft_kernel(
    const cplx<T>* __restrict__ U, cplx<T>* __restrict__ bvec, const T* __restrict__ dec,
    const cplx<T>* __restrict__ tw, int twlen, int M, int logM, int p, int L, int P2, int ldu,
    float* __restrict__ bscale) {
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* u = reinterpret_cast<cplx<T>*>(smem_raw);   // M (padded)
    const int m = blockIdx.x;
    const int b = blockIdx.y;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int H = M >> 1;
    const bool odd = (m & 1) != 0;
    const cplx<T>* src = U + ((int64_t)b * (L + 1) + m) * ldu;
    cplx<T>* out = bvec + ((int64_t)b * (p + 1) + m) * 2 * P2;
    // grid value t: the half grid, mirrored with the sign (-1)^m past M/2
    auto ld = [&](int t) {
        if (t <= H) return src[t];
        const cplx<T> v = src[M - t];
        return odd ? mk<T>(-v.r, -v.i) : v;
    };
    // mode j <= p: deconvolve and store as a right-hand side
    float mx = 0.f;   // largest magnitude stored (for bscale)
    auto st = [&](int j, cplx<T> v) {
        if (j > p) return;
        v = scale(v, dec[j]);
        if (odd) v = mk<T>(T(-0.5) * v.i, T(0.5) * v.r);
        out[(j & 1) * P2 + (j >> 1)] = v;
        mx = fmaxf(mx, fmaxf(fabsf((float)v.r), fabsf((float)v.i)));
    };
    if (logM >= 5) {
        block_fft_io<T, E>(u, logM, tw, twlen, ld, st);
    } else {
        for (int t = tid; t < M; t += nt) u[pad(t)] = ld(t);
        __syncthreads();
        block_fft_pad<T, E>(u, logM, tw, twlen, false);
        for (int j = tid; j < M; j += nt) st(j, u[pad(j)]);
    }
    if (tid == 0) out[P2 + (P2 - 1)] = mk<T>(T(0), T(0));
    if (bscale) {   // the column's largest magnitude, for the FP16 operator kernel
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0) atomicMax(reinterpret_cast<int*>(bscale) + (int64_t)b * (L + 1) + m, __float_as_int(mx));
    }
}

template <class T>
void launch_spread(const hpx_plan_s* P, cudaStream_t s) {
    const auto& g = P->g;
    const auto& t = P->t;
    const int H = g.M / 2;
    constexpr int EW = 12, DM = 4, NS = 4;
    if (sizeof(T) == 4 && t.spreadH <= EW && t.spreadD <= DM) {
        // rows a block needs: its first window start .. the last window end
        const int nrw = t.spreadRows - t.spreadH + EW + DM;
        const size_t smem = (size_t)(32 * 33 + NS * 32 * nrw) * sizeof(cplx<float>);
        auto kern = spread_rb_kernel<EW, DM, NS>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dim3 grid((H + 32) / 32, g.B);
        kern<<<grid, 256, smem, s>>>((const cplx<float>*)P->Y, (cplx<float>*)P->U, t.hstart, (const float*)t.hwts,
                                     t.spreadH, H, g.p, g.Q, g.L, P->ldu, nrw);
        return;
    }
    const size_t smem = (size_t)(32 * 33 + 32 * t.spreadRows) * sizeof(cplx<T>);
    cudaFuncSetAttribute(spread_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((H + 32) / 32, (g.L + 32) / 32, g.B);
    spread_kernel<T><<<grid, 256, smem, s>>>((const cplx<T>*)P->Y, (cplx<T>*)P->U, t.hstart, (const T*)t.hwts,
                                             t.spreadH, H, g.p, g.Q, g.L, P->ldu);
}

// lat_fft_pair_kernel: the same outputs for two orders per block, one M-point
// FFT for both.  The grid of an even order m is symmetric (u[M-t] = u[t]), that
// of the odd order m+1 antisymmetric, so the transform Z of their sum splits as
//     B_m(j) = (Z_j + Z_{M-j}) / 2,   B_{m+1}(j) = (Z_j - Z_{M-j}) / 2,
// and only the modes j <= p and j >= M - p of Z are kept (in shared memory).
template <class T, int E>
__global__ void __launch_bounds__(512, (E <= 16 ? 2 : 1)) lat_fft_pair_kernel(
    const cplx<T>* __restrict__ U, cplx<T>* __restrict__ bvec, const T* __restrict__ dec,
    const cplx<T>* __restrict__ tw, int twlen, int M, int logM, int p, int L, int P2, int ldu,
    float* __restrict__ bscale) {
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* u = reinterpret_cast<cplx<T>*>(smem_raw);   // M (padded)
    cplx<T>* zlo = u + M + M / 16;                         // Z_j, j = 0..p
    cplx<T>* zhi = zlo + (p + 1);                          // Z_{M-j}, j = 0..p
    const int m0 = 2 * blockIdx.x, m1 = m0 + 1;
    const int b = blockIdx.y;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int H = M >> 1;
    const bool has1 = m1 <= L;
    const cplx<T>* s0 = U + ((int64_t)b * (L + 1) + m0) * ldu;
    const cplx<T>* s1 = U + ((int64_t)b * (L + 1) + (has1 ? m1 : m0)) * ldu;
    auto ld = [&](int t) {
        const bool lo = t <= H;
        const int tt = lo ? t : M - t;
        cplx<T> v = s0[tt];
        if (has1) {
            const cplx<T> w = s1[tt];
            v = lo ? add(v, w) : sub(v, w);
        }
        return v;
    };
    auto st = [&](int j, cplx<T> v) {
        if (j <= p) zlo[j] = v;
        else if (j >= M - p) zhi[M - j] = v;
    };
    block_fft_io<T, E>(u, logM, tw, twlen, ld, st);
    __syncthreads();
    cplx<T>* out0 = bvec + ((int64_t)b * (p + 1) + m0) * 2 * P2;
    cplx<T>* out1 = out0 + 2 * P2;
    float mx0 = 0.f, mx1 = 0.f;   // largest magnitudes stored (for bscale)
    for (int j = tid; j <= p; j += nt) {
        const cplx<T> a = zlo[j], c = (j == 0) ? zlo[0] : zhi[j];
        const T dj = dec[j];
        const cplx<T> v0 = scale(add(a, c), T(0.5) * dj);
        out0[(j & 1) * P2 + (j >> 1)] = v0;
        mx0 = fmaxf(mx0, fmaxf(fabsf((float)v0.r), fabsf((float)v0.i)));
        if (has1) {
            const cplx<T> v = scale(sub(a, c), T(0.5) * dj);   // B_{m+1}(j), times i/2 below
            out1[(j & 1) * P2 + (j >> 1)] = mk<T>(T(-0.5) * v.i, T(0.5) * v.r);
            mx1 = fmaxf(mx1, 0.5f * fmaxf(fabsf((float)v.r), fabsf((float)v.i)));
        }
    }
    if (tid == 0) {
        out0[P2 + (P2 - 1)] = mk<T>(T(0), T(0));
        if (has1) out1[P2 + (P2 - 1)] = mk<T>(T(0), T(0));
    }
    if (bscale) {   // the columns' largest magnitudes, for the FP16 operator kernel
        for (int o = 16; o > 0; o >>= 1) {
            mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, o));
            mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, o));
        }
        if ((tid & 31) == 0) {   // non-negative floats order like their bits
            atomicMax(reinterpret_cast<int*>(bscale) + (int64_t)b * (L + 1) + m0, __float_as_int(mx0));
            if (has1) atomicMax(reinterpret_cast<int*>(bscale) + (int64_t)b * (L + 1) + m1, __float_as_int(mx1));
        }
    }
}

// lat_fft_pair_kernel with the grid length M = 2^LOGM fixed at compile time
// (fft_ct.cuh).
//
// FP32 precision at the highest latitude modes: an FP32 FFT leaves every
// output with an absolute error of about 2^-24 times the norm of its input,
// which for a smooth grid (a steep spectrum: most of the power at low latitude
// frequencies) swamps the small modes near j = p that carry the highest
// degrees.  The FP32 kernel therefore transforms the leaky first difference
// dz_t = z_t - rho z_{t-1} (cyclic, rho = 7/8, one rounding: a fused
// multiply-add), whose norm is mostly that of the grid's high-frequency part,
// and recovers Z_j = DFT(dz)_j / (1 - rho e^{-2 pi i j / M}).  The division is
// exact algebra; it amplifies rounding errors by at most 1 / (1 - rho) = 8 at
// j = 0 (a rough grid, e.g. white noise, loses up to a factor of about 5 there),
// while a smooth grid keeps the high modes about ten times more accurately.
constexpr float kPrewhiten = 0.875f;

// 1 / (1 - rho e^{-2 pi i j / M}) for 0 <= j < M, without cancellation:
// 1 - rho e^{-i x} = (1 - rho) + 2 rho sin^2(x/2) + i rho sin x.
template <int M>
__device__ __forceinline__ cplx<float> prewhiten_inverse(int j) {
    float sn, cs;
    sincospif((float)j / (float)M, &sn, &cs);   // sin, cos of x/2, x = 2 pi j / M
    const float a = (1.f - kPrewhiten) + 2.f * kPrewhiten * sn * sn;
    const float b = 2.f * kPrewhiten * sn * cs;
    const float inv = 1.f / (a * a + b * b);
    return mk<float>(a * inv, -b * inv);
}

template <class T, int LOGM, int NT>
__global__ void __launch_bounds__(NT, ((1 << LOGM) / NT == 16 ? (LOGM <= 13 ? 1024 / NT : 1) : 512 / NT)) lat_fft_pair_ct_kernel(
    const cplx<T>* __restrict__ U, cplx<T>* __restrict__ bvec, const T* __restrict__ dec,
    const cplx<T>* __restrict__ tw, int twlen, int p, int L, int P2, int ldu, float* __restrict__ bscale,
    unsigned char* __restrict__ bpk) {
    constexpr int M = 1 << LOGM;
    constexpr int H = M >> 1;
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* u = reinterpret_cast<cplx<T>*>(smem_raw);   // M (padded)
    cplx<T>* zlo = u + M + M / 16;                         // Z_j, j = 0..p
    cplx<T>* zhi = zlo + (p + 1);                          // Z_{M-j}, j = 0..p
    // blocks of one pair of orders and consecutive maps run together (map
    // index fastest), so the packed b of a pair's 32 maps, which share every
    // 128-byte line of the B layout, is written while its lines are in L2
    const int b = blockIdx.x;
    const int m0 = 2 * blockIdx.y, m1 = m0 + 1;
    const int tid = threadIdx.x;
    const bool has1 = m1 <= L;
    const cplx<T>* s0 = U + ((int64_t)b * (L + 1) + m0) * ldu;
    const cplx<T>* s1 = U + ((int64_t)b * (L + 1) + (has1 ? m1 : m0)) * ldu;
    auto ld = [&](int t, int) {
        const bool lo = t <= H;
        const int tt = lo ? t : M - t;
        cplx<T> v = s0[tt];
        if (has1) {
            const cplx<T> w = s1[tt];
            v = lo ? add(v, w) : sub(v, w);
        }
        return v;
    };
    if constexpr (sizeof(T) == 4) {
        // transform dz_t = z_t - rho z_{t-1}, then divide by 1 - rho e^{-2 pi i j / M}
        auto ldw = [&](int t, int pi) {
            const cplx<T> z = ld(t, pi), zp = ld((t + M - 1) & (M - 1), pi);
            return mk<T>(fmaf(-kPrewhiten, zp.r, z.r), fmaf(-kPrewhiten, zp.i, z.i));
        };
        auto stw = [&](int j, int, cplx<T> v) {
            if (j <= p) zlo[j] = mul(v, prewhiten_inverse<M>(j));
            else if (j >= M - p) zhi[M - j] = mul(v, conjg(prewhiten_inverse<M>(M - j)));
        };
        ct::fft<T, LOGM, NT, false, false>(u, tw, twlen >> LOGM, ldw, stw);
    } else {
        auto st = [&](int j, int, cplx<T> v) {
            if (j <= p) zlo[j] = v;
            else if (j >= M - p) zhi[M - j] = v;
        };
        ct::fft<T, LOGM, NT, false, false>(u, tw, twlen >> LOGM, ld, st);
    }
    if constexpr (sizeof(T) == 4) {
        if (bpk) {   // FP16 pairs for the tensor cores, scaled per column by its largest magnitude
            __shared__ float2 red32[32];
            // B_m(j) and i/2 B_{m+1}(j) (the values of the bvec form below) by
            // (column, parity of j, k = j >> 1) into the FFT buffer, which is free
            // now; one spare slot every 8 k, so that the packing below, where
            // lane g reads k = 8 g + e, spreads over the banks
            cplx<float>* vb = u;
            const int LD = P2 + (P2 >> 3) + 1;
            auto vidx = [&](int col, int par, int k) { return (col * 2 + par) * LD + k + (k >> 3); };
            float mx0 = 0.f, mx1 = 0.f;
            for (int j = tid; j <= p; j += NT) {
                const cplx<float> a = zlo[j], c = (j == 0) ? zlo[0] : zhi[j];
                const float dj = dec[j];
                const cplx<float> v0 = scale(add(a, c), 0.5f * dj);
                vb[vidx(0, j & 1, j >> 1)] = v0;
                mx0 = fmaxf(mx0, fmaxf(fabsf(v0.r), fabsf(v0.i)));
                if (has1) {
                    const cplx<float> v = scale(sub(a, c), 0.5f * dj);
                    const cplx<float> v1 = mk<float>(-0.5f * v.i, 0.5f * v.r);
                    vb[vidx(1, j & 1, j >> 1)] = v1;
                    mx1 = fmaxf(mx1, fmaxf(fabsf(v1.r), fabsf(v1.i)));
                }
            }
            const float2 mx = block_max2(make_float2(mx0, mx1), red32);   // (its barrier also publishes vb)
            mx0 = mx.x;
            mx1 = mx.y;
            if (tid == 0) {
                bscale[(int64_t)b * (L + 1) + m0] = mx0;
                if (has1) bscale[(int64_t)b * (L + 1) + m1] = mx1;
            }
            auto val = [&](int col, int par, int k) {   // zero past the column
                return (k < P2 && 2 * k + par <= p) ? vb[vidx(col, par, k)] : mk<float>(0.f, 0.f);
            };
            pack_column(bpk, b, m0, L, P2, pow2_scale(mx0, 13), [&](int par, int k) { return val(0, par, k); },
                        tid, NT);
            if (has1)
                pack_column(bpk, b, m1, L, P2, pow2_scale(mx1, 13), [&](int par, int k) { return val(1, par, k); },
                            tid, NT);
            return;
        }
    }
    cplx<T>* out0 = bvec + ((int64_t)b * (p + 1) + m0) * 2 * P2;
    cplx<T>* out1 = out0 + 2 * P2;
    float mx0 = 0.f, mx1 = 0.f;   // largest magnitudes stored (for bscale)
    for (int j = tid; j <= p; j += NT) {
        const cplx<T> a = zlo[j], c = (j == 0) ? zlo[0] : zhi[j];
        const T dj = dec[j];
        const cplx<T> v0 = scale(add(a, c), T(0.5) * dj);
        out0[(j & 1) * P2 + (j >> 1)] = v0;
        mx0 = fmaxf(mx0, fmaxf(fabsf((float)v0.r), fabsf((float)v0.i)));
        if (has1) {
            const cplx<T> v = scale(sub(a, c), T(0.5) * dj);   // B_{m+1}(j), times i/2 below
            out1[(j & 1) * P2 + (j >> 1)] = mk<T>(T(-0.5) * v.i, T(0.5) * v.r);
            mx1 = fmaxf(mx1, 0.5f * fmaxf(fabsf((float)v.r), fabsf((float)v.i)));
        }
    }
    if (tid == 0) {
        out0[P2 + (P2 - 1)] = mk<T>(T(0), T(0));
        if (has1) out1[P2 + (P2 - 1)] = mk<T>(T(0), T(0));
    }
    if (bscale) {   // the columns' largest magnitudes, for the FP16 operator kernel
        for (int o = 16; o > 0; o >>= 1) {
            mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, o));
            mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, o));
        }
        if ((tid & 31) == 0) {   // non-negative floats order like their bits
            atomicMax(reinterpret_cast<int*>(bscale) + (int64_t)b * (L + 1) + m0, __float_as_int(mx0));
            if (has1) atomicMax(reinterpret_cast<int*>(bscale) + (int64_t)b * (L + 1) + m1, __float_as_int(mx1));
        }
    }
}

// The packed form of b (fp16pair.cuh) from bvec and the column maxima in
// bscale: one block of 256 threads per (map tile, order, parity), two K-chunks
// per step; thread = (chunk, group of 8 k, map), so that the 8 lanes of a
// 128-byte line of the packed layout are adjacent in a warp (full-line stores)
// and each thread reads 64 contiguous bytes of its map's column.
__global__ void __launch_bounds__(256) pack_b_tiles_kernel(const cplx<float>* __restrict__ bvec,
                                                           unsigned char* __restrict__ bpk,
                                                           const float* __restrict__ bscale, int p, int L, int P2,
                                                           int B) {
    const int m = blockIdx.x, par = blockIdx.y, mt = blockIdx.z;
    const int nch = (P2 + 31) >> 5;
    const int t = threadIdx.x, n = t & 31, kg = (t >> 5) & 3, cl = t >> 7;
    const int b = mt * 32 + n;
    if (b >= B) return;   // columns past the batch stay zero
    const float sc = pow2_scale(bscale[(int64_t)b * (L + 1) + m], 13);
    const cplx<float>* col = bvec + (((int64_t)b * (p + 1) + m) * 2 + par) * P2;
    unsigned char* half = packed_half(bpk, b, m, par, L, nch);
    const int offr = packed_col_offset(b);
    for (int ch = cl; ch < nch; ch += 2) {
        const int g8 = ch * 4 + kg;
        pack_group(half, offr, g8, sc, [&](int k) { return k < P2 ? col[k] : mk<float>(0.f, 0.f); });
    }
}

bool packs_b(const hpx_plan_s* P) {
    return P->bpk && P->precision == HPX_FP32 && ((P->fusedM && P->use_tc) || (!P->fusedM && P->dTC));
}

template <class T>
void launch_lat_fft(const hpx_plan_s* P, cudaStream_t s, bool packed) {
    const auto& g = P->g;
    packed = packed && sizeof(T) == 4 && P->bpk && P->bscale;
    // packed b: either written by the compile-time grid-FFT kernel itself, or
    // (P->packSep, and the other grid lengths) FP32 b with the column maxima as
    // atomic maxima of the float bits, then one pass of pack_b_tiles_kernel
    int logM = 0;
    while ((1 << logM) < g.M) ++logM;
    const bool inFft = packed && !P->packSep && logM >= 12 && logM <= 14;
    if (packed && !inFft) cudaMemsetAsync(P->bscale, 0, (size_t)g.B * (g.L + 1) * sizeof(float), s);
    float* bsc = packed ? P->bscale : nullptr;
    auto pack_pass = [&]() {
        if (packed && !inFft)
            pack_b_tiles_kernel<<<dim3(g.L + 1, 2, (g.B + 31) / 32), 256, 0, s>>>(
                (const cplx<float>*)P->bvec, P->bpk, P->bscale, g.p, g.L, g.P2, g.B);
    };
    const size_t smem = (size_t)(g.M + g.M / 16) * sizeof(cplx<T>);
    if (logM >= 12 && logM <= 14) {   // two orders per block, compile-time grid length
        const size_t smem2 = (size_t)(g.M + g.M / 16 + 2 * (g.p + 1)) * sizeof(cplx<T>);
        dim3 grid2(g.B, (g.L + 2) / 2);
        auto run = [&](auto kern, int threads) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
            kern<<<grid2, threads, smem2, s>>>((const cplx<T>*)P->U, (cplx<T>*)P->bvec, (const T*)P->t.dec,
                                               (const cplx<T>*)P->t.twid, g.Lmax, g.p, g.L, g.P2, P->ldu,
                                               bsc, inFft ? P->bpk : nullptr);
        };
        const bool e32 = P->latE == 32;   // elements per thread (the plan's tuning), else 16
        if (logM == 12) { if (e32) run(lat_fft_pair_ct_kernel<T, 12, 128>, 128); else run(lat_fft_pair_ct_kernel<T, 12, 256>, 256); }
        else if (logM == 13) { if (e32) run(lat_fft_pair_ct_kernel<T, 13, 256>, 256); else run(lat_fft_pair_ct_kernel<T, 13, 512>, 512); }
        else run(lat_fft_pair_ct_kernel<T, 14, 512>, 512);
        pack_pass();
        return;
    }
    if (logM >= 5) {   // two orders per block
        const size_t smem2 = (size_t)(g.M + g.M / 16 + 2 * (g.p + 1)) * sizeof(cplx<T>);
        auto kern2 = g.M > 16 * 512 ? lat_fft_pair_kernel<T, 32> : lat_fft_pair_kernel<T, 16>;
        cudaFuncSetAttribute(kern2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
        dim3 grid2((g.L + 2) / 2, g.B);
        kern2<<<grid2, 512, smem2, s>>>((const cplx<T>*)P->U, (cplx<T>*)P->bvec, (const T*)P->t.dec,
                                        (const cplx<T>*)P->t.twid, g.Lmax, g.M, logM, g.p, g.L, g.P2, P->ldu,
                                        bsc);
    } else {
        auto kern = g.M > 16 * 512 ? lat_fft_kernel<T, 32> : lat_fft_kernel<T, 16>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dim3 grid(g.L + 1, g.B);
        kern<<<grid, 512, smem, s>>>((const cplx<T>*)P->U, (cplx<T>*)P->bvec, (const T*)P->t.dec,
                                     (const cplx<T>*)P->t.twid, g.Lmax, g.M, logM, g.p, g.L, g.P2, P->ldu, bsc);
    }
    pack_pass();
}

template void launch_spread<float>(const hpx_plan_s*, cudaStream_t);
template void launch_spread<double>(const hpx_plan_s*, cudaStream_t);
template void launch_lat_fft<float>(const hpx_plan_s*, cudaStream_t, bool);
template void launch_lat_fft<double>(const hpx_plan_s*, cudaStream_t, bool);

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
