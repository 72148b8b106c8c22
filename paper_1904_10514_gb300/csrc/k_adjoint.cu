// The exact adjoint (transpose) of the analysis, hpx_synthesize: every stage of
// Algorithm 1 transposed and applied in reverse order.  Inner products: plain
// sum_i f_i g_i on maps, plain Re(x conj y) on the intermediate complex arrays,
// and sum_l [Re(a_l0 conj b_l0) + 2 sum_{m>0} Re(a_lm conj b_lm)] on alm (so the
// input alm are weighted by 1 at m = 0 and 2 at m > 0 first).  The analysis
// returns real a_l0 and a_l^p, so the imaginary parts of those inputs are
// dropped, as the exact transpose of a real-valued output does.
//
//   rot_adj    transposed Givens sweeps (Sec. 3.3): each sweep appends a zero
//              carry and applies the rotations in reverse order, top down; the
//              sweeps run in reverse order as a register wavefront.
//   dense_adj  beta -> b:  D^T (latitude least squares and Legendre change of basis)
//   nufft_adj  b -> y: deconvolution, inverse M-point FFT and interpolation from the
//              fine grid to the DFS nodes (the transposed ES spreading, Sec. 3.2.2)
//   ring_adj   y -> ring samples: transposed shift/Nyquist/padding and inverse
//              DFT per ring pair (Sec. 3.1)
//   pole_adj   adds the transposed pole fit (Sec. 3.2.1) to the 3 rings per cap
#include "fft_ct.cuh"
#include "plan.h"
#include "plan_math.h"
#include "sweep.cuh"

namespace hpx {

// ---------------------------------------------------------------- rot_adj
// One transposed pass of K sweeps.  The chain has n_in elements on entry and
// n_in + K on exit.  Stage k (undoing the pass's forward stage K-1-k) handles
// rotation index i = n_in + 2k - t at time t, from the top of its chain down:
//     (carry, out_i) = (c_i a - s_i carry, s_i a + c_i carry),  a = input w_{i-1},
// then emits the carry as out_0 at i = 0.  Idle slots hold (0, 0) (clearing the
// carry before the stage starts) and the emission slot holds (1, 0).
template <class T, int K>
__device__ __forceinline__ void sweep_pass_adj(T* chain, int64_t ldc, int n_in, const cplx<T>* __restrict__ A,
                                               int coff) {
    T carry[K], pipe[K];
#pragma unroll
    for (int k = 0; k < K; ++k) { carry[k] = T(0); pipe[k] = T(0); }
    const int steps = n_in + 2 * K - 1;
    for (int t = 0; t < steps; ++t) {
        const T x0 = (t < n_in) ? chain[(int64_t)(n_in - 1 - t) * ldc] : T(0);
        const cplx<T>* row = A + (int64_t)t * 32 + coff;
#pragma unroll
        for (int k = K - 1; k >= 0; --k) {
            const T x = (k == 0) ? x0 : pipe[k - 1];
            const cplx<T> cs = row[k];
            const T o = cs.i * x + cs.r * carry[k];
            carry[k] = cs.r * x - cs.i * carry[k];
            pipe[k] = o;
        }
        const int j = n_in + 2 * K - 2 - t;
        if (j >= 0 && j < n_in + K) chain[(int64_t)j * ldc] = pipe[K - 1];
    }
}

template <class T, int KMAX>
__global__ void __launch_bounds__(128) rot_adj_kernel(const T* __restrict__ alm, T* __restrict__ beta2,
                                                      const int64_t* __restrict__ skOff,
                                                      const cplx<T>* __restrict__ skewT, int nq, int P2, int L,
                                                      int p, int B, int64_t nalm, int ngroups, int nitems,
                                                      T wpos, bool dropim) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nitems) return;
    const int g = warp % ngroups;
    const int c = (warp / ngroups) & 1;
    const int m = L - warp / (2 * ngroups);
    const int m0 = m & 1;
    const int S = (m - m0) >> 1;
    const int ncol = 2 * B;
    const int col = 32 * g + lane;
    if (col >= ncol) return;
    const int par = (m0 + c) & 1;
    const int q0 = (m0 == 1 && c == 1) ? 1 : 0;
    T* chain = beta2 + (((int64_t)m * 2 + par) * P2 + q0) * ncol + col;
    const int64_t ldc = ncol;
    // order-m chain from the weighted input coefficients
    int n = chain_len(m, c, L);
    const int b = col >> 1, ri = col & 1;
    const T w = (m == 0) ? T(1) : wpos;
    const bool drop = dropim && ri == 1 && (m == 0 || m == p);
    const T* in = alm + (int64_t)b * nalm * 2 + ri;
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2 + m + c;
    for (int i = 0; i < n; ++i) chain[(int64_t)i * ldc] = drop ? T(0) : w * in[(base + 2 * i) * 2];
    // forward passes: F full passes of KMAX at s = 0, KMAX, ..., then the binary
    // digits of the remainder r (16, 8, 4, 2, 1 below KMAX); undo them in reverse.
    const int F = S / KMAX, r = S % KMAX;
    auto block = [&](int s_lo, int K) {
        const int e = 32 - (s_lo & 31) - K;
        return skewT + (skOff[(size_t)(m0 * 2 + c) * nq + (s_lo >> 5)] + e) * 32;
    };
    auto coff = [&](int s_lo, int K) { return 32 - (s_lo & 31) - K; };
#define HPX_SUBPASS_ADJ(KK)                                                               \
    if (KK < KMAX && (r & KK)) {                                                          \
        const int s_lo = F * KMAX + (r & ~(2 * KK - 1));                                  \
        sweep_pass_adj<T, KK>(chain, ldc, n, block(s_lo, KK), coff(s_lo, KK));          \
        n += KK;                                                                          \
    }
    HPX_SUBPASS_ADJ(1)
    HPX_SUBPASS_ADJ(2)
    HPX_SUBPASS_ADJ(4)
    HPX_SUBPASS_ADJ(8)
    HPX_SUBPASS_ADJ(16)
#undef HPX_SUBPASS_ADJ
    for (int f = F - 1; f >= 0; --f) {
        const int s_lo = f * KMAX;
        sweep_pass_adj<T, KMAX>(chain, ldc, n, block(s_lo, KMAX), coff(s_lo, KMAX));
        n += KMAX;
    }
}

// FP32: the same transposed pass with the angle rows and the chain inputs of
// step t staged through a per-warp ring of shared memory RB - 1 steps ahead
// (8-byte copies of the 32 angles, one 4-byte copy per lane).  Every lane of
// the warp runs it (lanes without a column neither load nor store chain values).
// The outputs go to indices above every input still to be read, so the
// prefetch never reads a value this pass has rewritten.
template <int K, int RB>
__device__ __forceinline__ void sweep_pass_adj_staged(float* chain, int64_t ldc, int n_in, bool live,
                                                      const cplx<float>* __restrict__ A, int coff,
                                                      cplx<float>* ring) {
    constexpr int SL = SweepRing<RB>::kSlot;
    const int lane = threadIdx.x & 31;
    float carry[K], pipe[K];
#pragma unroll
    for (int k = 0; k < K; ++k) { carry[k] = 0.f; pipe[k] = 0.f; }
    const int steps = n_in + 2 * K - 1;
    auto issue = [&](int t) {
        if (t < steps) {
            cplx<float>* slot = ring + (t % RB) * SL;
            cp_async8(slot + lane, A + (int64_t)t * 32 + lane, 8);
            const bool have = live && t < n_in;
            cp_async4(reinterpret_cast<float*>(slot + 32) + lane,
                      have ? chain + (int64_t)(n_in - 1 - t) * ldc : (const float*)A, have ? 4 : 0);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
#pragma unroll
    for (int q = 0; q < RB - 1; ++q) issue(q);
    for (int t = 0; t < steps; ++t) {
        __syncwarp();
        issue(t + RB - 1);
        asm volatile("cp.async.wait_group %0;" ::"n"(RB - 1) : "memory");
        __syncwarp();
        const cplx<float>* slot = ring + (t % RB) * SL;
        const float x0 = reinterpret_cast<const float*>(slot + 32)[lane];
        const cplx<float>* row = slot + coff;
#pragma unroll
        for (int k = K - 1; k >= 0; --k) {
            const float x = (k == 0) ? x0 : pipe[k - 1];
            const cplx<float> cs = row[k];
            const float o = cs.i * x + cs.r * carry[k];
            carry[k] = cs.r * x - cs.i * carry[k];
            pipe[k] = o;
        }
        const int j = n_in + 2 * K - 2 - t;
        if (live && j >= 0 && j < n_in + K) chain[(int64_t)j * ldc] = pipe[K - 1];
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
}

// rot_adj_kernel for FP32 with the staged passes (one real column per lane,
// warps of 2 per block; the whole warp stays in the passes).
template <int KMAX>
__global__ void __launch_bounds__(64, 8) rot_adj_staged_kernel(const float* __restrict__ alm, float* __restrict__ beta2,
                                                              const int64_t* __restrict__ skOff,
                                                              const cplx<float>* __restrict__ skewT, int nq, int P2,
                                                              int L, int p, int B, int64_t nalm, int ngroups,
                                                              int nitems, float wpos, bool dropim) {
    constexpr int RB = 8;
    constexpr int SL = SweepRing<RB>::kSlot;
    __shared__ __align__(16) cplx<float> rings[2][RB * SL];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nitems) return;   // whole warps leave together
    cplx<float>* ring = rings[(threadIdx.x >> 5) & 1];
    const int g = warp % ngroups;
    const int c = (warp / ngroups) & 1;
    const int m = L - warp / (2 * ngroups);
    const int m0 = m & 1;
    const int S = (m - m0) >> 1;
    const int ncol = 2 * B;
    const int col = 32 * g + lane;
    const bool live = col < ncol;
    const int par = (m0 + c) & 1;
    const int q0 = (m0 == 1 && c == 1) ? 1 : 0;
    float* chain = beta2 + (((int64_t)m * 2 + par) * P2 + q0) * ncol + (live ? col : 0);
    const int64_t ldc = ncol;
    int n = chain_len(m, c, L);
    if (live) {   // order-m chain from the weighted input coefficients
        const int b = col >> 1, ri = col & 1;
        const float w = (m == 0) ? 1.f : wpos;
        const bool drop = dropim && ri == 1 && (m == 0 || m == p);
        const float* in = alm + (int64_t)b * nalm * 2 + ri;
        const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2 + m + c;
        for (int i = 0; i < n; ++i) chain[(int64_t)i * ldc] = drop ? 0.f : w * in[(base + 2 * i) * 2];
    }
    __syncwarp();
    const int F = S / KMAX, r = S % KMAX;
    auto block = [&](int s_lo, int K) {
        const int e = 32 - (s_lo & 31) - K;
        return skewT + (skOff[(size_t)(m0 * 2 + c) * nq + (s_lo >> 5)] + e) * 32;
    };
    auto coff = [&](int s_lo, int K) { return 32 - (s_lo & 31) - K; };
#define HPX_SUBPASS_ADJ(KK)                                                                        \
    if (KK < KMAX && (r & KK)) {                                                                   \
        const int s_lo = F * KMAX + (r & ~(2 * KK - 1));                                           \
        sweep_pass_adj_staged<KK, RB>(chain, ldc, n, live, block(s_lo, KK), coff(s_lo, KK), ring); \
        n += KK;                                                                                   \
    }
    HPX_SUBPASS_ADJ(1)
    HPX_SUBPASS_ADJ(2)
    HPX_SUBPASS_ADJ(4)
    HPX_SUBPASS_ADJ(8)
    HPX_SUBPASS_ADJ(16)
#undef HPX_SUBPASS_ADJ
    for (int f = F - 1; f >= 0; --f) {
        const int s_lo = f * KMAX;
        sweep_pass_adj_staged<KMAX, RB>(chain, ldc, n, live, block(s_lo, KMAX), coff(s_lo, KMAX), ring);
        n += KMAX;
    }
}

// ---------------------------------------------------------------- dense_adj
namespace {
constexpr int AK = 64;   // output rows (k) per block
constexpr int AC = 32;   // columns (m, map) per block
constexpr int AQ = 16;   // reduction chunk (q)
}  // namespace

template <class T>
__global__ void __launch_bounds__(256) dense_adj_kernel(const T* __restrict__ D, const cplx<T>* __restrict__ beta,
                                                        cplx<T>* __restrict__ bvec, int P2, int p, int L, int B) {
    __shared__ T Ds[AQ][AK + 1];
    __shared__ cplx<T> Bs[AQ][AC];
    const int mpar = blockIdx.z >> 1, par = blockIdx.z & 1;
    const int nmp = (L >= mpar) ? (L - mpar) / 2 + 1 : 0;
    const int ncols = nmp * B;
    const int c0 = blockIdx.x * AC, k0 = blockIdx.y * AK;
    if (c0 >= ncols) return;
    const T* Dm = D + ((size_t)(mpar * 2 + par) * P2) * P2;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    T accr[4][2], acci[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 2; ++c) { accr[a][c] = T(0); acci[a][c] = T(0); }
    for (int qb = 0; qb < P2; qb += AQ) {
        for (int e = tid; e < AQ * AK; e += 256) {
            const int qq = e / AK, kk = e % AK;
            const int q = qb + qq, k = k0 + kk;
            Ds[qq][kk] = (q < P2 && k < P2) ? Dm[(size_t)q * P2 + k] : T(0);
        }
        for (int e = tid; e < AQ * AC; e += 256) {
            const int qq = e / AC, cc = e % AC;
            const int q = qb + qq, col = c0 + cc;
            const int l = 2 * q + par;
            cplx<T> v = mk<T>(T(0), T(0));
            if (col < ncols && q < P2 && l <= L && l >= mpar) {
                const int b = col % B, mi = col / B;
                const int m = 2 * mi + mpar;
                v = beta[(((int64_t)m * 2 + par) * P2 + q) * B + b];
            }
            Bs[qq][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int qq = 0; qq < AQ; ++qq) {
            T a[4];
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) a[rr] = Ds[qq][tx * 4 + rr];
            cplx<T> bb[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) bb[c] = Bs[qq][ty * 2 + c];
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    accr[rr][c] += a[rr] * bb[c].r;
                    acci[rr][c] += a[rr] * bb[c].i;
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
        cplx<T>* out = bvec + (((int64_t)b * (p + 1) + m) * 2 + par) * P2;
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int k = k0 + tx * 4 + rr;
            if (k < P2) out[k] = mk<T>(accr[rr][c], acci[rr][c]);
        }
    }
}

// ---------------------------------------------------------------- nufft_adj
template <class T>
__global__ void __launch_bounds__(512) nufft_adj_kernel(const cplx<T>* __restrict__ bvec, cplx<T>* __restrict__ Y,
                                                        const int* __restrict__ nrowptr,
                                                        const int* __restrict__ nent, const T* __restrict__ nentw,
                                                        const T* __restrict__ dec, const cplx<T>* __restrict__ tw,
                                                        int twlen, int M, int logM, int p, int Q, int P2) {
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* u = reinterpret_cast<cplx<T>*>(smem_raw);
    const int m = blockIdx.x, b = blockIdx.y;
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool odd = (m & 1) != 0;
    const cplx<T>* in = bvec + ((int64_t)b * (p + 1) + m) * 2 * P2;
    for (int j = tid; j < M; j += nt) {
        cplx<T> v = mk<T>(T(0), T(0));
        if (j <= p) {
            v = in[(j & 1) * P2 + (j >> 1)];
            if (odd) v = mk<T>(T(0.5) * v.i, T(-0.5) * v.r);   // conj(i/2) v
            v = scale(v, dec[j]);
        }
        u[j] = v;
    }
    __syncthreads();
    block_fft(u, M, logM, tw, twlen, true);
    cplx<T>* out = Y + (int64_t)b * Q * (p + 1) + m;
    for (int r = tid; r < Q; r += nt) {
        T ar = T(0), ai = T(0);
        const int e1 = nrowptr[r + 1];
        for (int e = nrowptr[r]; e < e1; ++e) {
            const int code = nent[e];
            const int t = code & ((1 << 30) - 1);
            T w = nentw[e];
            if (odd && (code >> 30)) w = -w;
            const cplx<T> v = u[t];
            ar += w * v.r;
            ai += w * v.i;
        }
        out[(int64_t)r * (p + 1)] = mk<T>(ar, ai);
    }
}

// ---------------------------------------------------------------- ring_adj
template <class T>
__global__ void __launch_bounds__(256) ring_adj_kernel(
    const cplx<T>* __restrict__ Y, T* __restrict__ maps, const int* __restrict__ nphi_t,
    const int* __restrict__ startN_t, const int* __restrict__ startS_t, const int* __restrict__ pow2_t,
    const int* __restrict__ logn_t, const int* __restrict__ fftL_t, const int* __restrict__ logL_t,
    const int64_t* __restrict__ shOff_t, const int64_t* __restrict__ chOff_t, const int64_t* __restrict__ bhOff_t,
    const cplx<T>* __restrict__ shift, const cplx<T>* __restrict__ chirp, const cplx<T>* __restrict__ bhat,
    const cplx<T>* __restrict__ tw, int twlen, int p, int Q, int64_t npix, int npairs,
    const int* __restrict__ ringlist) {
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
    const int i = ringlist ? ringlist[blockIdx.x] : npairs - 1 - (int)blockIdx.x;
    const int b = blockIdx.y;
    const int n = nphi_t[i], h = n >> 1;
    const int sN = startN_t[i], sS = startS_t[i];
    const bool equator = (sN == sS);
    const int tid = threadIdx.x, nt = blockDim.x;
    const cplx<T>* ph = shift + shOff_t[i];
    const cplx<T>* rowN = Y + ((int64_t)b * Q + (i + 1)) * (p + 1);
    const cplx<T>* rowS = Y + ((int64_t)b * Q + (Q - 2 - i)) * (p + 1);
    const bool bl = !pow2_t[i];
    const cplx<T>* ch = chirp + chOff_t[i];
    // X = H_N + i H_S with H the Hermitian extension of z_m = conj(ph_m) y_m
    for (int m = tid; m <= h; m += nt) {
        const cplx<T> w = conjg(ph[m]);
        const cplx<T> zn = mul(w, rowN[m]);
        const cplx<T> zs = equator ? mk<T>(T(0), T(0)) : mul(w, rowS[m]);
        cplx<T> xm, xc;
        if (m == 0 || m == h) {
            xm = mk<T>(zn.r, zs.r);
        } else {
            xm = mk<T>(T(0.5) * (zn.r - zs.i), T(0.5) * (zn.i + zs.r));   // zn/2 + i zs/2
            xc = mk<T>(T(0.5) * (zn.r + zs.i), T(0.5) * (-zn.i + zs.r));  // conj(zn)/2 + i conj(zs)/2
        }
        // Bluestein: transform conj(X) forward, premultiplied by the chirp
        if (bl) {
            buf[m] = mul(conjg(xm), ch[m]);
            if (m != 0 && m != h) buf[n - m] = mul(conjg(xc), ch[n - m]);
        } else {
            buf[m] = xm;
            if (m != 0 && m != h) buf[n - m] = xc;
        }
    }
    if (bl) {
        const int L = fftL_t[i];
        for (int k = n + tid; k < L; k += nt) buf[k] = mk<T>(T(0), T(0));
        __syncthreads();
        const cplx<T>* bh = bhat + bhOff_t[i];
        block_fft(buf, L, logL_t[i], tw, twlen, false);
        for (int k = tid; k < L; k += nt) buf[k] = mul(buf[k], bh[k]);
        __syncthreads();
        block_fft(buf, L, logL_t[i], tw, twlen, true);
        for (int k = tid; k < n; k += nt) buf[k] = conjg(mul(buf[k], ch[k]));
        __syncthreads();
    } else {
        __syncthreads();
        block_fft(buf, n, logn_t[i], tw, twlen, true);
    }
    T* f = maps + (int64_t)b * npix;
    for (int k = tid; k < n; k += nt) {
        f[sN + k] = buf[k].r;
        if (!equator) f[sS + k] = buf[k].i;
    }
}

template <class T>
__global__ void pole_adj_kernel(const cplx<T>* __restrict__ Y, T* __restrict__ maps, const int* __restrict__ poleN,
                                const int* __restrict__ poleS, const double* __restrict__ w, int npole, int p,
                                int Q, int64_t npix) {
    const int b = blockIdx.x;
    const cplx<T>* Yb = Y + (int64_t)b * Q * (p + 1);
    const T vn = Yb[0].r;
    const T vs = Yb[(int64_t)(Q - 1) * (p + 1)].r;
    T* f = maps + (int64_t)b * npix;
    for (int k = threadIdx.x; k < npole; k += blockDim.x) {
        f[poleN[k]] += (T)w[k] * vn;
        f[poleS[k]] += (T)w[k] * vs;
    }
}

// ring_adj_kernel for the ring classes of 4096 points and more, with the
// compile-time FFT: the first pass reads the Hermitian extension X of each ring
// pair straight from the rows of Y.
template <class T, int LOGN, int NT, bool BLUE>
__global__ void __launch_bounds__(NT, (LOGN <= 13 ? 1024 / NT : 1)) ring_adj_ct_kernel(
    const cplx<T>* __restrict__ Y, T* __restrict__ maps, const int* __restrict__ nphi_t,
    const int* __restrict__ startN_t, const int* __restrict__ startS_t, const int64_t* __restrict__ shOff_t,
    const int64_t* __restrict__ chOff_t, const int64_t* __restrict__ bhOff_t, const cplx<T>* __restrict__ shift,
    const cplx<T>* __restrict__ chirp, const cplx<T>* __restrict__ bhat, const cplx<T>* __restrict__ tw, int twlen,
    int p, int Q, int64_t npix, const int* __restrict__ ringlist) {
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
    const int i = ringlist[blockIdx.y];
    const int b = blockIdx.x;
    const int n = nphi_t[i], h = n >> 1;
    const int sN = startN_t[i], sS = startS_t[i];
    const bool equator = (sN == sS);
    const int tid = threadIdx.x;
    const int twstep = twlen >> LOGN;
    const cplx<T>* ph = shift + shOff_t[i];
    const cplx<T>* rowN = Y + ((int64_t)b * Q + (i + 1)) * (p + 1);
    const cplx<T>* rowS = Y + ((int64_t)b * Q + (Q - 2 - i)) * (p + 1);
    // X_k = H_N + i H_S, H the Hermitian extension of z_m = conj(ph_m) y_m (k < n)
    auto X = [&](int k) {
        const int m = k <= h ? k : n - k;
        const cplx<T> w = conjg(ph[m]);
        const cplx<T> zn = mul(w, rowN[m]);
        const cplx<T> zs = equator ? mk<T>(T(0), T(0)) : mul(w, rowS[m]);
        if (m == 0 || m == h) return mk<T>(zn.r, zs.r);
        if (k <= h) return mk<T>(T(0.5) * (zn.r - zs.i), T(0.5) * (zn.i + zs.r));   // zn/2 + i zs/2
        return mk<T>(T(0.5) * (zn.r + zs.i), T(0.5) * (-zn.i + zs.r));              // conj(zn)/2 + i conj(zs)/2
    };
    auto to_smem = [&](int, int pi, cplx<T> v) { buf[pi] = v; };
    if constexpr (!BLUE) {
        ct::fft<T, LOGN, NT, true, false>(buf, tw, twstep, [&](int k, int) { return X(k); }, to_smem);
    } else {
        // inverse DFT of length n via Bluestein: transform conj(X) forward with the chirp
        const cplx<T>* ch = chirp + chOff_t[i];
        const cplx<T>* bh = bhat + bhOff_t[i];
        ct::fft<T, LOGN, NT, false, false>(
            buf, tw, twstep, [&](int k, int) { return k < n ? mul(conjg(X(k)), ch[k]) : mk<T>(T(0), T(0)); },
            [&](int j, int pi, cplx<T> v) { buf[pi] = mul(v, bh[j]); });
        ct::fft<T, LOGN, NT, true, true>(
            buf, tw, twstep, [&](int, int pi) { return buf[pi]; },
            [&](int j, int pi, cplx<T> v) { buf[pi] = j < n ? conjg(mul(v, ch[j])) : v; });
    }
    T* f = maps + (int64_t)b * npix;
    for (int k = tid; k < n; k += NT) {
        const cplx<T> v = buf[ct::padc(k)];
        f[sN + k] = v.r;
        if (!equator) f[sS + k] = v.i;
    }
}

template <class T>
void launch_ring_adj(const hpx_plan_s* P, T* maps, cudaStream_t s) {
    const auto& g = P->g;
    const auto& t = P->t;
    auto old = [&](int blocks, size_t smem, const int* list) {
        cudaFuncSetAttribute(ring_adj_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dim3 grid(blocks, g.B);
        ring_adj_kernel<T><<<grid, 256, smem, s>>>(
            (const cplx<T>*)P->Y, maps, t.nphi, t.startN, t.startS, t.pow2, t.logn, t.fftL, t.logL, t.shOff,
            t.chOff, t.bhOff, (const cplx<T>*)t.shift, (const cplx<T>*)t.chirp, (const cplx<T>*)t.bhat,
            (const cplx<T>*)t.twid, g.Lmax, g.p, g.Q, g.npix, g.npairs, list);
    };
    if (!P->ringList) {
        old(g.npairs, (size_t)g.smem_ring * sizeof(cplx<T>), nullptr);
        return;
    }
    for (const auto& c : P->ringClasses) {
        if (c.N < kRingCtMin) {
            old(c.count, (size_t)c.N * sizeof(cplx<T>), P->ringList + c.first);
            continue;
        }
        const size_t smem = (size_t)(c.N + c.N / 16) * sizeof(cplx<T>);
        dim3 grid(g.B, c.count);
        auto run = [&](auto kern, int threads) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kern<<<grid, threads, smem, s>>>((const cplx<T>*)P->Y, maps, t.nphi, t.startN, t.startS, t.shOff,
                                             t.chOff, t.bhOff, (const cplx<T>*)t.shift, (const cplx<T>*)t.chirp,
                                             (const cplx<T>*)t.bhat, (const cplx<T>*)t.twid, g.Lmax, g.p, g.Q,
                                             g.npix, P->ringList + c.first);
        };
        if (c.N == 4096) {
            if (c.blue) run(ring_adj_ct_kernel<T, 12, 256, true>, 256);
            else run(ring_adj_ct_kernel<T, 12, 256, false>, 256);
        } else if (c.N == 8192) {
            if (c.blue) run(ring_adj_ct_kernel<T, 13, 512, true>, 512);
            else run(ring_adj_ct_kernel<T, 13, 512, false>, 512);
        } else {
            if (c.blue) run(ring_adj_ct_kernel<T, 14, 512, true>, 512);
            else run(ring_adj_ct_kernel<T, 14, 512, false>, 512);
        }
    }
}

template <class T>
void launch_adjoint(const hpx_plan_s* P, const T* alm, T* maps, cudaStream_t s, T wpos) {
    const auto& g = P->g;
    const auto& t = P->t;
    {
        const int ngroups = (2 * g.B + 31) / 32;
        const int nitems = (g.L + 1) * 2 * ngroups;
        const int blocks = (nitems * 32 + 127) / 128;
        constexpr int KMAX = sizeof(T) == 4 ? 32 : 16;
        if constexpr (sizeof(T) == 4)   // angle rows and inputs staged ahead of use
            rot_adj_staged_kernel<32><<<(nitems * 32 + 63) / 64, 64, 0, s>>>(
                (const float*)alm, (float*)P->beta, t.skOff, (const cplx<float>*)t.skewT, t.nq, g.P2, g.L, g.p, g.B,
                g.nalm, ngroups, nitems, (float)wpos, true);
        else
            rot_adj_kernel<T, KMAX><<<blocks, 128, 0, s>>>(alm, (T*)P->beta, t.skOff, (const cplx<T>*)t.skewT, t.nq,
                                                           g.P2, g.L, g.p, g.B, g.nalm, ngroups, nitems, wpos, true);
    }
    {
        const int nmp = g.L / 2 + 1;
        dim3 grid((nmp * g.B + AC - 1) / AC, (g.P2 + AK - 1) / AK, 4);
        dense_adj_kernel<T><<<grid, 256, 0, s>>>((const T*)t.D, (const cplx<T>*)P->beta, (cplx<T>*)P->bvec, g.P2,
                                                 g.p, g.L, g.B);
    }
    {
        int logM = 0;
        while ((1 << logM) < g.M) ++logM;
        const size_t smem = (size_t)g.M * sizeof(cplx<T>);
        cudaFuncSetAttribute(nufft_adj_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        // columns m > lmax carry no coefficients: their rows of Y are zero
        cudaMemsetAsync(P->Y, 0, (size_t)g.B * g.Q * (g.p + 1) * sizeof(cplx<T>), s);
        dim3 grid(g.L + 1, g.B);
        if (!launch_nufft2(P, s))
            nufft_adj_kernel<T><<<grid, 512, smem, s>>>((const cplx<T>*)P->bvec, (cplx<T>*)P->Y, t.nrowptr, t.nent,
                                                    (const T*)t.nentw, (const T*)t.dec, (const cplx<T>*)t.twid,
                                                    g.Lmax, g.M, logM, g.p, g.Q, g.P2);
    }
    {
        launch_ring_adj<T>(P, maps, s);
        pole_adj_kernel<T><<<g.B, 128, 0, s>>>((const cplx<T>*)P->Y, maps, t.poleN, t.poleS, t.polew, t.npole,
                                               g.p, g.Q, g.npix);
    }
}

// ---------------------------------------------------------------- synthesis
// Spherical-harmonic synthesis f(pixel) = sum_{l,m} a_l^m Y_l^m (real maps: m < 0
// from a_l^{-m} = (-1)^m conj(a_l^m)), the inverse direction of the analysis:
//   1. the transposed Givens sweeps (rot_adj_kernel, unweighted) take order m to
//      order-0/1 Legendre coefficients (the sweeps are orthogonal: R^-1 = R^T);
//   2. dense_adj_kernel with the table Es maps those to the coefficients X_j of
//      F_m(t) = (1/sqrt(2 pi)) sum_l a_l^m Pbar_l^m(cos t) = sum_j X_j cos|sin(j t);
//   3. nufft_adj_kernel evaluates the cosine / sine series at the latitude nodes
//      (type-2 NUFFT; for even m it returns w_r F_m(t_r) with w_r = 2 on rings);
//   4. ring_synth_kernel folds the orders into the nphi frequencies of each ring,
//      F_m e^{i m phi0} summed over m = n mod nphi (m in [-lmax, lmax]), and
//      transforms back to the ring's pixels (N and S rings packed as one complex
//      sequence; Bluestein for the polar rings).
template <class T>
__global__ void __launch_bounds__(256) ring_synth_kernel(
    const cplx<T>* __restrict__ Y, T* __restrict__ maps, const int* __restrict__ nphi_t,
    const int* __restrict__ startN_t, const int* __restrict__ startS_t, const int* __restrict__ shifted_t,
    const int* __restrict__ pow2_t, const int* __restrict__ logn_t, const int* __restrict__ fftL_t,
    const int* __restrict__ logL_t, const int64_t* __restrict__ chOff_t, const int64_t* __restrict__ bhOff_t,
    const cplx<T>* __restrict__ chirp, const cplx<T>* __restrict__ bhat, const cplx<T>* __restrict__ tw, int twlen,
    int p, int L, int Q, int64_t npix, int npairs, const int* __restrict__ ringlist) {
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
    const int i = ringlist ? ringlist[blockIdx.x] : npairs - 1 - (int)blockIdx.x;
    const int b = blockIdx.y;
    const int n = nphi_t[i];
    const int sN = startN_t[i], sS = startS_t[i];
    const bool equator = (sN == sS);
    const int sh = shifted_t[i];
    const int tid = threadIdx.x, nt = blockDim.x;
    const cplx<T>* rowN = Y + ((int64_t)b * Q + (i + 1)) * (p + 1);
    const cplx<T>* rowS = Y + ((int64_t)b * Q + (Q - 2 - i)) * (p + 1);
    const bool bl = !pow2_t[i];
    const cplx<T>* ch = chirp + chOff_t[i];
    // G_m = F_m e^{i m phi0}, phi0 = sh pi / n; F_m = Y / 2 for even m (ring weight 2)
    auto G = [&](const cplx<T>* row, int m) {
        cplx<T> v = row[m];
        if (!(m & 1)) v = scale(v, T(0.5));
        if (m == 0) return mk<T>(v.r, T(0));
        if (!sh) return v;
        const int r = m % (2 * n);
        T sn, cs;
        if (sizeof(T) == 4) {
            float a, c;
            sincospif((float)r / (float)n, &a, &c);
            sn = (T)a; cs = (T)c;
        } else {
            double a, c;
            sincospi((double)r / (double)n, &a, &c);
            sn = (T)a; cs = (T)c;
        }
        return mul(v, mk<T>(cs, sn));
    };
    for (int k = tid; k < n; k += nt) {
        cplx<T> cN = mk<T>(T(0), T(0)), cS = cN;
        for (int m = k; m <= L; m += n) {   // m = k + q n >= 0
            cN = add(cN, G(rowN, m));
            if (!equator) cS = add(cS, G(rowS, m));
        }
        for (int m = n - k; m <= L; m += n) {   // -m = k - q n < 0: G_{-m} = conj(G_m)
            if (m == 0) continue;
            cN = add(cN, conjg(G(rowN, m)));
            if (!equator) cS = add(cS, conjg(G(rowS, m)));
        }
        // z = cN + i cS; the forward transform runs on conj(z) = (cN.r - cS.i) - i (cN.i + cS.r)
        const cplx<T> zconj = mk<T>(cN.r - cS.i, -(cN.i + cS.r));
        buf[k] = bl ? mul(zconj, ch[k]) : zconj;
    }
    if (bl) {
        const int Lb = fftL_t[i];
        for (int k = n + tid; k < Lb; k += nt) buf[k] = mk<T>(T(0), T(0));
        __syncthreads();
        const cplx<T>* bh = bhat + bhOff_t[i];
        block_fft(buf, Lb, logL_t[i], tw, twlen, false);
        for (int k = tid; k < Lb; k += nt) buf[k] = mul(buf[k], bh[k]);
        __syncthreads();
        block_fft(buf, Lb, logL_t[i], tw, twlen, true);
        for (int k = tid; k < n; k += nt) buf[k] = mul(buf[k], ch[k]);
        __syncthreads();
    } else {
        __syncthreads();
        block_fft(buf, n, logn_t[i], tw, twlen, false);
    }
    // Z = conj(DFT(conj z)): north = Re Z, south = Im Z = -Im DFT(conj z)
    T* f = maps + (int64_t)b * npix;
    for (int k = tid; k < n; k += nt) {
        f[sN + k] = buf[k].r;
        if (!equator) f[sS + k] = -buf[k].i;
    }
}

// ring_synth_kernel for the launches of one transform length N = 2^LOGN >= 4096
// (the ring classes of the analysis: N = nphi for plain rings, the Bluestein
// convolution length otherwise) with the compile-time FFT of fft_ct.cuh: the
// fold of the orders is the first pass's input and the pixels are written from
// shared memory after the transform.
template <class T, int LOGN, int NT, bool BLUE>
__global__ void __launch_bounds__(NT, (LOGN <= 13 ? 1024 / NT : 1)) ring_synth_ct_kernel(
    const cplx<T>* __restrict__ Y, T* __restrict__ maps, const int* __restrict__ nphi_t,
    const int* __restrict__ startN_t, const int* __restrict__ startS_t, const int* __restrict__ shifted_t,
    const int64_t* __restrict__ chOff_t, const int64_t* __restrict__ bhOff_t, const cplx<T>* __restrict__ chirp,
    const cplx<T>* __restrict__ bhat, const cplx<T>* __restrict__ tw, int twlen, int p, int L, int Q,
    int64_t npix, const int* __restrict__ ringlist) {
    const int twstep = twlen >> LOGN;
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
    const int i = ringlist[blockIdx.y];
    const int b = blockIdx.x;
    const int n = nphi_t[i];
    const int sN = startN_t[i], sS = startS_t[i];
    const bool equator = (sN == sS);
    const int sh = shifted_t[i];
    const int tid = threadIdx.x;
    const cplx<T>* rowN = Y + ((int64_t)b * Q + (i + 1)) * (p + 1);
    const cplx<T>* rowS = Y + ((int64_t)b * Q + (Q - 2 - i)) * (p + 1);
    // G_m = F_m e^{i m phi0}, phi0 = sh pi / n; F_m = Y / 2 for even m (ring weight 2)
    auto G = [&](const cplx<T>* row, int m) {
        cplx<T> v = row[m];
        if (!(m & 1)) v = scale(v, T(0.5));
        if (m == 0) return mk<T>(v.r, T(0));
        if (!sh) return v;
        const int r = m % (2 * n);
        T sn, cs;
        if constexpr (sizeof(T) == 4) {
            sincospif((float)r / (float)n, &sn, &cs);
        } else {
            sincospi((double)r / (double)n, &sn, &cs);
        }
        return mul(v, mk<T>(cs, sn));
    };
    // conj(z_k), z = (folded north) + i (folded south)
    auto fold = [&](int k) {
        cplx<T> cN = mk<T>(T(0), T(0)), cS = cN;
        for (int m = k; m <= L; m += n) {
            cN = add(cN, G(rowN, m));
            if (!equator) cS = add(cS, G(rowS, m));
        }
        for (int m = n - k; m <= L; m += n) {
            if (m == 0) continue;
            cN = add(cN, conjg(G(rowN, m)));
            if (!equator) cS = add(cS, conjg(G(rowS, m)));
        }
        return mk<T>(cN.r - cS.i, -(cN.i + cS.r));
    };
    auto to_smem = [&](int, int pi, cplx<T> v) { buf[pi] = v; };
    if constexpr (!BLUE) {
        ct::fft<T, LOGN, NT, false, false>(buf, tw, twstep, [&](int k, int) { return fold(k); }, to_smem);
    } else {
        const cplx<T>* ch = chirp + chOff_t[i];
        const cplx<T>* bh = bhat + bhOff_t[i];
        ct::fft<T, LOGN, NT, false, false>(
            buf, tw, twstep, [&](int k, int) { return k < n ? mul(fold(k), ch[k]) : mk<T>(T(0), T(0)); },
            [&](int j, int pi, cplx<T> v) { buf[pi] = mul(v, bh[j]); });
        ct::fft<T, LOGN, NT, true, true>(
            buf, tw, twstep, [&](int, int pi) { return buf[pi]; },
            [&](int j, int pi, cplx<T> v) { buf[pi] = j < n ? mul(v, ch[j]) : v; });
    }
    // Z = conj(DFT(conj z)): north = Re Z, south = Im Z = -Im DFT(conj z)
    T* f = maps + (int64_t)b * npix;
    for (int k = tid; k < n; k += NT) {
        const cplx<T> v = buf[ct::padc(k)];
        f[sN + k] = v.r;
        if (!equator) f[sS + k] = -v.i;
    }
}

template <class T>
void launch_ring_synth(const hpx_plan_s* P, T* maps, cudaStream_t s) {
    const auto& g = P->g;
    const auto& t = P->t;
    auto old = [&](int blocks, size_t smem, const int* list) {
        cudaFuncSetAttribute(ring_synth_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dim3 grid(blocks, g.B);
        ring_synth_kernel<T><<<grid, 256, smem, s>>>(
            (const cplx<T>*)P->Y, maps, t.nphi, t.startN, t.startS, t.shifted, t.pow2, t.logn, t.fftL, t.logL,
            t.chOff, t.bhOff, (const cplx<T>*)t.chirp, (const cplx<T>*)t.bhat, (const cplx<T>*)t.twid, g.Lmax, g.p,
            g.L, g.Q, g.npix, g.npairs, list);
    };
    if (!P->ringList) {
        old(g.npairs, (size_t)g.smem_ring * sizeof(cplx<T>), nullptr);
        return;
    }
    for (const auto& c : P->ringClasses) {
        if (c.N < kRingCtMin) {   // short rings: the radix-2 kernel, sized for the class's longest transform
            old(c.count, (size_t)c.N * sizeof(cplx<T>), P->ringList + c.first);
            continue;
        }
        const size_t smem = (size_t)(c.N + c.N / 16) * sizeof(cplx<T>);
        dim3 grid(g.B, c.count);
        auto run = [&](auto kern, int threads) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kern<<<grid, threads, smem, s>>>((const cplx<T>*)P->Y, maps, t.nphi, t.startN, t.startS, t.shifted,
                                             t.chOff, t.bhOff, (const cplx<T>*)t.chirp, (const cplx<T>*)t.bhat,
                                             (const cplx<T>*)t.twid, g.Lmax, g.p, g.L, g.Q, g.npix,
                                             P->ringList + c.first);
        };
        if (c.N == 4096) {
            if (c.blue) run(ring_synth_ct_kernel<T, 12, 256, true>, 256);
            else run(ring_synth_ct_kernel<T, 12, 256, false>, 256);
        } else if (c.N == 8192) {
            if (c.blue) run(ring_synth_ct_kernel<T, 13, 512, true>, 512);
            else run(ring_synth_ct_kernel<T, 13, 512, false>, 512);
        } else {
            if (c.blue) run(ring_synth_ct_kernel<T, 14, 512, true>, 512);
            else run(ring_synth_ct_kernel<T, 14, 512, false>, 512);
        }
    }
}

template <class T>
void launch_sh_synthesis(const hpx_plan_s* P, const T* alm, T* maps, cudaStream_t s, cudaEvent_t* ev) {
    const auto& g = P->g;
    const auto& t = P->t;
    if (ev) cudaEventRecord(ev[0], s);
    if (sizeof(T) == 4 && P->synT) {
        launch_synth_tc(P, (const float*)alm, s);   // the same operators on the tensor cores
    } else if (P->synM) {
        launch_synth_apply<T>(P, alm, s);   // the sweeps and Es composed per (m, c)
    } else {
        const int ngroups = (2 * g.B + 31) / 32;
        const int nitems = (g.L + 1) * 2 * ngroups;
        const int blocks = (nitems * 32 + 127) / 128;
        constexpr int KMAX = sizeof(T) == 4 ? 32 : 16;
        if constexpr (sizeof(T) == 4)
            rot_adj_staged_kernel<32><<<(nitems * 32 + 63) / 64, 64, 0, s>>>(
                (const float*)alm, (float*)P->beta, t.skOff, (const cplx<float>*)t.skewT, t.nq, g.P2, g.L, g.p, g.B,
                g.nalm, ngroups, nitems, 1.f, false);
        else
            rot_adj_kernel<T, KMAX><<<blocks, 128, 0, s>>>(alm, (T*)P->beta, t.skOff, (const cplx<T>*)t.skewT, t.nq,
                                                           g.P2, g.L, g.p, g.B, g.nalm, ngroups, nitems, T(1), false);
        const int nmp = g.L / 2 + 1;
        dim3 grid((nmp * g.B + AC - 1) / AC, (g.P2 + AK - 1) / AK, 4);
        dense_adj_kernel<T><<<grid, 256, 0, s>>>((const T*)t.Es, (const cplx<T>*)P->beta, (cplx<T>*)P->bvec, g.P2,
                                                 g.p, g.L, g.B);
    }
    if (ev) cudaEventRecord(ev[1], s);
    {
        int logM = 0;
        while ((1 << logM) < g.M) ++logM;
        const size_t smem = (size_t)g.M * sizeof(cplx<T>);
        cudaFuncSetAttribute(nufft_adj_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dim3 grid(g.L + 1, g.B);
        if (!launch_nufft2(P, s))
            nufft_adj_kernel<T><<<grid, 512, smem, s>>>((const cplx<T>*)P->bvec, (cplx<T>*)P->Y, t.nrowptr, t.nent,
                                                        (const T*)t.nentw, (const T*)t.dec, (const cplx<T>*)t.twid,
                                                        g.Lmax, g.M, logM, g.p, g.Q, g.P2);
    }
    if (ev) cudaEventRecord(ev[2], s);
    launch_ring_synth<T>(P, maps, s);
    if (ev)
        for (int k = 3; k <= hpx_plan_s::kStages; ++k) cudaEventRecord(ev[k], s);
}

template void launch_sh_synthesis<float>(const hpx_plan_s*, const float*, float*, cudaStream_t, cudaEvent_t*);
template void launch_sh_synthesis<double>(const hpx_plan_s*, const double*, double*, cudaStream_t, cudaEvent_t*);

template void launch_adjoint<float>(const hpx_plan_s*, const float*, float*, cudaStream_t, float);
template void launch_adjoint<double>(const hpx_plan_s*, const double*, double*, cudaStream_t, double);

}  // namespace hpx
