// Step 1 of Algorithm 1 (Sec. 3.1): per-ring trigonometric interpolation,
// half-pixel shift and zero padding, and the pole values of Sec. 3.2.1.
//
// One thread block handles one north/south ring pair of one map; the blocks of
// one ring pair for all maps are adjacent in the grid, so the ring's tables stay
// in L2 while its maps are processed.  The two real rings (same nphi, same first
// longitude) are packed into one complex sequence z = f_N + i f_S and
// transformed once:
//   * nphi a power of two: Stockham FFT of length nphi in shared memory;
//   * otherwise (polar rings 4j): Bluestein's chirp-z transform with a
//     power-of-two convolution length L >= 2 nphi - 1; the chirps and the
//     transformed conjugate chirp come from FP64-built tables.
// The interpolant coefficients of Eq. (trig_expansion) at the un-shifted
// longitudes of Eq. (upsamp) are then c_m = c~_m e^{-i m phi0} (Eq. interp_cond
// and the shift that follows it), with the Nyquist term split evenly between
// +-nphi/2 and zero padding for m > nphi/2 (the `shift` table folds 1/nphi,
// the phase and the Nyquist factor together).  Output row r of Y holds the
// coefficients m = 0..p of latitude node r (r = ring index + 1).
#include <algorithm>

#include "fft_ct.cuh"
#include "plan.h"

namespace hpx {

constexpr int kRingThreads = 512;

// Output rows of step 1 from the ring pair's DFT (z = DFT of f_N + i f_S, n
// points, element k at buf[pad(k)]).
//   ew == 0 (the analysis, Sec. 3.1): c_m = c~_m e^{-i m phi0} for m <= n/2 with the
//     Nyquist split, 0 above (table ph = (1/n) e^{-i m phi0} with that split folded in).
//   ew != 0 (the transpose of the synthesis' ring stage, used by the equal-weight
//     quadrature of Sec. 2.2): for every m <= L the ring's Fourier sum
//     D_m = sum_k f_k e^{-i m lambda_k} (m taken mod n, so the polar rings alias),
//     times ew and the weight of order m: the synthesis folds Y_m / 2 (even m) or
//     Y_m (odd m) at +-m, so the plain transpose carries 1 (even m > 0), 2 (odd m)
//     and 1/2 (m = 0); the transpose for the coefficient inner product with
//     weight 2 for m > 0 halves the m > 0 ones: 1/2 for even m, 1 for odd m.
//     0 for L < m <= p.
template <class T, class BUF>
__device__ __forceinline__ void ring_rows_out(BUF zat, int n, int p, int L, const cplx<T>* __restrict__ ph, bool sh,
                                              T ew, cplx<T>* rowN, cplx<T>* rowS, bool equator, int tid, int nt) {
    const int h = n >> 1;
    for (int m = tid; m <= p; m += nt) {
        cplx<T> cN = mk<T>(T(0), T(0)), cS = cN;
        if (ew == T(0) ? m <= h : m <= L) {
            const int k = m % n;
            const cplx<T> zm = zat(k);
            const cplx<T> zc = conjg(zat(k == 0 ? 0 : n - k));
            const cplx<T> fn = scale(add(zm, zc), T(0.5));              // n * c~_m (north)
            const cplx<T> d = sub(zm, zc);
            const cplx<T> fs = mk<T>(T(0.5) * d.i, T(-0.5) * d.r);      // n * c~_m (south)
            cplx<T> w;
            if (ew == T(0)) {
                w = ph[m];
            } else {
                const T wm = ew * ((m & 1) ? T(1) : T(0.5));
                if (sh) {   // e^{-i m pi / n}
                    T sn, cs;
                    if constexpr (sizeof(T) == 4) sincospif(-(float)(m % (2 * n)) / (float)n, &sn, &cs);
                    else sincospi(-(double)(m % (2 * n)) / (double)n, &sn, &cs);
                    w = mk<T>(wm * cs, wm * sn);
                } else {
                    w = mk<T>(wm, T(0));
                }
            }
            cN = mul(fn, w);
            cS = mul(fs, w);
        }
        rowN[m] = cN;
        if (!equator) rowS[m] = cS;
    }
}

// The same step for the launches of one transform length N = 2^LOGN >= 4096
// whose ring pairs are all of one kind (BLUE: Bluestein rings of convolution
// length N; else rings of N points): the FFT length, the thread count
// (N / 16 or N / 32) and the pass structure are compile-time constants
// (fft_ct.cuh), and the kind of ring is known, so neither transform carries
// the other's code.
template <class T, int LOGN, int NT, bool BLUE>
__global__ void __launch_bounds__(NT, ((1 << LOGN) / NT == 16 ? (LOGN <= 13 ? 1024 / NT : 1) : 512 / NT)) ring_ct_kernel(
    const T* __restrict__ maps, cplx<T>* __restrict__ Y, const int* __restrict__ nphi_t,
    const int* __restrict__ startN_t, const int* __restrict__ startS_t, const int64_t* __restrict__ shOff_t,
    const int64_t* __restrict__ chOff_t, const int64_t* __restrict__ bhOff_t, const cplx<T>* __restrict__ shift,
    const cplx<T>* __restrict__ chirp, const cplx<T>* __restrict__ bhat, const cplx<T>* __restrict__ tw, int twlen,
    int p, int Q, int64_t npix, const int* __restrict__ ringlist, T ew, const int* __restrict__ shifted_t, int L,
    const int64_t* __restrict__ mapIdx) {
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
    const int i = ringlist[blockIdx.y];
    const int b = blockIdx.x;
    const int n = nphi_t[i];
    const int sN = startN_t[i], sS = startS_t[i];
    const bool equator = (sN == sS);
    const T* f = maps + (mapIdx ? mapIdx[b] : (int64_t)b * npix);
    const int tid = threadIdx.x;
    const int twstep = twlen >> LOGN;
    auto sample = [&](int k) { return mk<T>(f[sN + k], equator ? T(0) : f[sS + k]); };
    auto to_smem = [&](int, int pi, cplx<T> v) { buf[pi] = v; };
    if constexpr (!BLUE) {
        ct::fft<T, LOGN, NT, false, false>(buf, tw, twstep, [&](int k, int) { return sample(k); }, to_smem);
    } else {
        // Bluestein: chirped samples in, times the transformed kernel out; the
        // inverse transform applies the output chirp in its last pass
        const cplx<T>* ch = chirp + chOff_t[i];
        const cplx<T>* bh = bhat + bhOff_t[i];
        ct::fft<T, LOGN, NT, false, false>(
            buf, tw, twstep, [&](int k, int) { return k < n ? mul(sample(k), ch[k]) : mk<T>(T(0), T(0)); },
            [&](int j, int pi, cplx<T> v) { buf[pi] = mul(v, bh[j]); });
        ct::fft<T, LOGN, NT, true, true>(
            buf, tw, twstep, [&](int, int pi) { return buf[pi]; },
            [&](int j, int pi, cplx<T> v) { buf[pi] = j < n ? mul(v, ch[j]) : v; });
    }
    cplx<T>* rowN = Y + ((int64_t)b * Q + (i + 1)) * (p + 1);
    cplx<T>* rowS = Y + ((int64_t)b * Q + (Q - 2 - i)) * (p + 1);
    ring_rows_out<T>([&](int k) { return buf[ct::padc(k)]; }, n, p, L, shift + shOff_t[i], shifted_t[i] != 0, ew,
                     rowN, rowS, equator, tid, NT);
}

// A Bluestein ring of nphi = 4j points as four transforms of j points: with
// t = 4u + s the DFT is Z[q + r j] = sum_s (-i)^{s r} W^{s q} Y_s[q]
// (W = e^{-2 pi i / nphi}, q < j, r < 4), Y_s the DFT of the subsequence
// z[4u + s].  Each Y_s is a Bluestein convolution of L/4 = 2^(LOGN-2) points
// (L the ring's convolution length, L/4 >= 2j), run on NT/4 threads of the
// block beside the other three (compile-time FFT, one padded quarter of the
// buffer each): a quarter of the transformed-kernel table per ring and one
// radix-16 pass fewer than the full-length convolution.  The radix-4 step writes
// Z into the free tail of the quarters (quarter r, from slot padc(j)), and the
// output rows follow as in ring_ct_kernel.
template <class T, int LOGN, int NT>
__global__ void __launch_bounds__(NT, (LOGN <= 13 ? 1024 / NT : 1)) ring4_ct_kernel(
    const T* __restrict__ maps, cplx<T>* __restrict__ Y, const int* __restrict__ nphi_t,
    const int* __restrict__ startN_t, const int* __restrict__ startS_t, const int64_t* __restrict__ shOff_t,
    const int64_t* __restrict__ ch4Off_t, const int64_t* __restrict__ bh4Off_t, const cplx<T>* __restrict__ shift,
    const cplx<T>* __restrict__ chirp4, const cplx<T>* __restrict__ bhat4, const cplx<T>* __restrict__ tw, int twlen,
    int p, int Q, int64_t npix, const int* __restrict__ ringlist, T ew, const int* __restrict__ shifted_t, int L,
    const int64_t* __restrict__ mapIdx) {
    constexpr int LOGQ = LOGN - 2, NQ = 1 << LOGQ, NTQ = NT / 4;
    constexpr int QS = NQ + NQ / 16;   // one padded quarter
    static_assert(NTQ % 32 == 0, "ring4: whole warps per quarter");
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
    const int i = ringlist[blockIdx.y];
    const int b = blockIdx.x;
    const int n = nphi_t[i], jq = n >> 2;
    const int sN = startN_t[i], sS = startS_t[i];
    const T* f = maps + (mapIdx ? mapIdx[b] : (int64_t)b * npix);
    const int tid = threadIdx.x;
    const int s = tid / NTQ, ltid = tid - s * NTQ;
    cplx<T>* qb = buf + s * QS;
    const cplx<T>* ch = chirp4 + ch4Off_t[i];
    const cplx<T>* bh = bhat4 + bh4Off_t[i];
    const int twstep = twlen >> LOGQ;
    ct::fft<T, LOGQ, NTQ, false, false>(
        qb, tw, twstep,
        [&](int u, int) {
            return u < jq ? mul(mk<T>(f[sN + 4 * u + s], f[sS + 4 * u + s]), ch[u]) : mk<T>(T(0), T(0));
        },
        [&](int k, int pi, cplx<T> v) { qb[pi] = mul(v, bh[k]); }, ltid);
    ct::fft<T, LOGQ, NTQ, true, true>(
        qb, tw, twstep, [&](int, int pi) { return qb[pi]; },
        [&](int k, int pi, cplx<T> v) { qb[pi] = k < jq ? mul(v, ch[k]) : v; }, ltid);
    const int S0 = ct::padc(jq);   // first slot past the Y_s values (S0 + jq <= QS)
    for (int q = tid; q < jq; q += NT) {
        T sn, cs;
        if constexpr (sizeof(T) == 4) sincospif(-2.f * (float)q / (float)n, &sn, &cs);
        else sincospi(-2.0 * (double)q / (double)n, &sn, &cs);
        const cplx<T> w1 = mk<T>(cs, sn), w2 = mul(w1, w1), w3 = mul(w1, w2);
        const int pq = ct::padc(q);
        const cplx<T> t0 = buf[pq], t1 = mul(w1, buf[QS + pq]), t2 = mul(w2, buf[2 * QS + pq]),
                      t3 = mul(w3, buf[3 * QS + pq]);
        const cplx<T> a = add(t0, t2), bb = sub(t0, t2), c = add(t1, t3), d = sub(t1, t3);
        buf[S0 + q] = add(a, c);                                   // r = 0
        buf[QS + S0 + q] = mk<T>(bb.r + d.i, bb.i - d.r);          // r = 1: bb - i d
        buf[2 * QS + S0 + q] = sub(a, c);                          // r = 2
        buf[3 * QS + S0 + q] = mk<T>(bb.r - d.i, bb.i + d.r);      // r = 3: bb + i d
    }
    __syncthreads();
    cplx<T>* rowN = Y + ((int64_t)b * Q + (i + 1)) * (p + 1);
    cplx<T>* rowS = Y + ((int64_t)b * Q + (Q - 2 - i)) * (p + 1);
    ring_rows_out<T>(
        [&](int k) {
            const int r = (k >= jq) + (k >= 2 * jq) + (k >= 3 * jq);
            return buf[r * QS + S0 + (k - r * jq)];
        },
        n, p, L, shift + shOff_t[i], shifted_t[i] != 0, ew, rowN, rowS, false, tid, NT);
}

// The step for ring pair i of map b by the whole block (runtime transform
// length; the generic form behind ring_fft_kernel and ring_list_kernel).
template <class T, int E>
__device__ __forceinline__ void ring_pair(
    cplx<T>* buf, int i, int b, const T* __restrict__ maps, cplx<T>* __restrict__ Y, const int* __restrict__ nphi_t,
    const int* __restrict__ startN_t, const int* __restrict__ startS_t, const int* __restrict__ pow2_t,
    const int* __restrict__ logn_t, const int* __restrict__ fftL_t, const int* __restrict__ logL_t,
    const int64_t* __restrict__ shOff_t, const int64_t* __restrict__ chOff_t, const int64_t* __restrict__ bhOff_t,
    const cplx<T>* __restrict__ shift, const cplx<T>* __restrict__ chirp, const cplx<T>* __restrict__ bhat,
    const cplx<T>* __restrict__ tw, int twlen, int p, int Q, int64_t npix, T ew, const int* __restrict__ shifted_t,
    int L, const int64_t* __restrict__ mapIdx) {
    const int n = nphi_t[i];
    const int sN = startN_t[i], sS = startS_t[i];
    const bool equator = (sN == sS);
    const T* f = maps + (mapIdx ? mapIdx[b] : (int64_t)b * npix);
    const int tid = threadIdx.x, nt = blockDim.x;

    auto sample = [&](int k) { return mk<T>(f[sN + k], equator ? T(0) : f[sS + k]); };
    auto same = [](int, cplx<T> v) { return v; };
    if (pow2_t[i] && logn_t[i] >= 5) {
        // the first FFT pass reads the rings from the map
        block_fft_pad_io<T, E, false, false>(buf, logn_t[i], tw, twlen, sample, same);
    } else if (!pow2_t[i] && logL_t[i] >= 5) {
        // Bluestein: the forward transform reads the chirped samples and its last
        // pass multiplies by the transformed kernel; the inverse transform's last
        // pass applies the output chirp
        const int L = fftL_t[i];
        const cplx<T>* ch = chirp + chOff_t[i];
        const cplx<T>* bh = bhat + bhOff_t[i];
        auto chirped = [&](int k) { return k < n ? mul(sample(k), ch[k]) : mk<T>(T(0), T(0)); };
        auto kern = [&](int j, cplx<T> v) { return mul(v, bh[j]); };
        auto fromsmem = [&](int k) { return buf[pad(k)]; };
        auto unchirp = [&](int j, cplx<T> v) { return j < n ? mul(v, ch[j]) : v; };
        (void)L;
        block_fft_pad_io<T, E, false, false>(buf, logL_t[i], tw, twlen, chirped, kern);
        block_fft_pad_io<T, E, true, true>(buf, logL_t[i], tw, twlen, fromsmem, unchirp);
    } else if (pow2_t[i]) {
        for (int k = tid; k < n; k += nt) buf[pad(k)] = sample(k);
        __syncthreads();
        block_fft_pad<T, E>(buf, logn_t[i], tw, twlen, false);
    } else {
        const int L = fftL_t[i];
        const cplx<T>* ch = chirp + chOff_t[i];
        const cplx<T>* bh = bhat + bhOff_t[i];
        for (int k = tid; k < L; k += nt) {
            cplx<T> v = mk<T>(T(0), T(0));
            if (k < n) v = mul(mk<T>(f[sN + k], equator ? T(0) : f[sS + k]), ch[k]);
            buf[pad(k)] = v;
        }
        __syncthreads();
        block_fft_pad<T, E>(buf, logL_t[i], tw, twlen, false);
        for (int k = tid; k < L; k += nt) buf[pad(k)] = mul(buf[pad(k)], bh[k]);
        __syncthreads();
        block_fft_pad<T, E>(buf, logL_t[i], tw, twlen, true);
        for (int k = tid; k < n; k += nt) buf[pad(k)] = mul(buf[pad(k)], ch[k]);
        __syncthreads();
    }

    cplx<T>* rowN = Y + ((int64_t)b * Q + (i + 1)) * (p + 1);
    cplx<T>* rowS = Y + ((int64_t)b * Q + (Q - 2 - i)) * (p + 1);
    ring_rows_out<T>([&](int k) { return buf[pad(k)]; }, n, p, L, shift + shOff_t[i], shifted_t[i] != 0, ew, rowN,
                     rowS, equator, tid, nt);
}


template <class T, int E>
__global__ void __launch_bounds__(kRingThreads, (E <= 16 ? 2 : 1)) ring_fft_kernel(
    const T* __restrict__ maps, cplx<T>* __restrict__ Y, const int* __restrict__ nphi_t,
    const int* __restrict__ startN_t, const int* __restrict__ startS_t,
    const int* __restrict__ pow2_t, const int* __restrict__ logn_t, const int* __restrict__ fftL_t,
    const int* __restrict__ logL_t, const int64_t* __restrict__ shOff_t,
    const int64_t* __restrict__ chOff_t, const int64_t* __restrict__ bhOff_t,
    const cplx<T>* __restrict__ shift, const cplx<T>* __restrict__ chirp,
    const cplx<T>* __restrict__ bhat, const cplx<T>* __restrict__ tw, int twlen, int p, int Q,
    int64_t npix, int npairs, const int* __restrict__ ringlist, T ew, const int* __restrict__ shifted_t, int L,
    const int64_t* __restrict__ mapIdx) {
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
    // largest rings first: blockIdx.y = 0 is the equator
    const int i = ringlist ? ringlist[blockIdx.y] : npairs - 1 - (int)blockIdx.y;
    ring_pair<T, E>(buf, i, blockIdx.x, maps, Y, nphi_t, startN_t, startS_t, pow2_t, logn_t, fftL_t, logL_t, shOff_t,
                    chOff_t, bhOff_t, shift, chirp, bhat, tw, twlen, p, Q, npix, ew, shifted_t, L, mapIdx);
}

// The short-ring part of the ring stage of every sub-plan of an uneven batch
// in persistent launches: the blocks walk a work list of (sub-plan, ring pair,
// map) items with transforms shorter than kRingCtMin points, built at plan time
// with the longest transforms first, in strides of the grid size; the
// sub-plans' tables and workspaces come from the job table.  The maps are read
// from the caller's array: those of a sub-plan whose maps are adjacent at the
// job's element offset from maps_base, the others at their own offsets (the
// job's mapIdx table).  NT
// threads per block (16 elements per thread): 128 for the items of 1024 and
// 2048 points, 32 for the shorter ones, each group its own launch.  The
// longer transforms run in the sub-plans' compile-time kernels.
template <class T, int NT>
__global__ void __launch_bounds__(NT, (NT == 32 ? 16 : 8)) ring_list_kernel(const RingJob<T>* __restrict__ jobs,
                                                                          const int4* __restrict__ items,
                                                                          int nitems, const T* __restrict__ maps_base) {
    extern __shared__ unsigned char smem_raw[];
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 w = items[it];
        const RingJob<T>& J = jobs[w.x];
        ring_pair<T, 16>(buf, w.y, w.z, maps_base + J.mapoff, J.Y, J.nphi, J.startN, J.startS, J.pow2, J.logn,
                         J.fftL, J.logL, J.shOff, J.chOff, J.bhOff, J.shift, J.chirp, J.bhat, J.tw, J.twlen, J.p, J.Q,
                         J.npix, T(0), J.shifted, J.L, J.mapIdx);
        __syncthreads();   // the next item overwrites the shared buffer
    }
}

template <class T>
void launch_ring_list(const RingJob<T>* jobs, const int4* items, int nitems, int nlong, const T* maps_base,
                      cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto run = [&](auto kern, int threads, int maxN, const int4* first, int n, int perSM) {
        if (n <= 0) return;
        const size_t smem = (size_t)(maxN + maxN / 16) * sizeof(cplx<T>);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<std::min(n, sms * perSM), threads, smem, s>>>(jobs, first, n, maps_base);
    };
    // items [0, nlong): 1024 or 2048 points; [nlong, nitems): 512 or fewer
    run(ring_list_kernel<T, 128>, 128, 2048, items, nlong, 8);
    run(ring_list_kernel<T, 32>, 32, 512, items + nlong, nitems - nlong, 16);
}

template void launch_ring_list<float>(const RingJob<float>*, const int4*, int, int, const float*, cudaStream_t);
template void launch_ring_list<double>(const RingJob<double>*, const int4*, int, int, const double*, cudaStream_t);

// Pole values (Sec. 3.2.1): a fixed linear functional of the samples of the
// three rings nearest each pole (unit-weight quadratic least squares in the
// tangent plane, built at plan time).  Row 0 / row Q-1 of Y: the value at
// m = 0, zero for m > 0.
template <class T>
__global__ void pole_kernel(const T* __restrict__ maps, cplx<T>* __restrict__ Y,
                            const int* __restrict__ poleN, const int* __restrict__ poleS,
                            const double* __restrict__ w, int npole, int p, int Q, int64_t npix,
                            const int64_t* __restrict__ mapIdx) {
    const int b = blockIdx.x;
    const T* f = maps + (mapIdx ? mapIdx[b] : (int64_t)b * npix);
    __shared__ double red[2][32];
    double sn = 0.0, ss = 0.0;
    for (int k = threadIdx.x; k < npole; k += blockDim.x) {
        sn += w[k] * (double)f[poleN[k]];
        ss += w[k] * (double)f[poleS[k]];
    }
    for (int o = 16; o > 0; o >>= 1) {
        sn += __shfl_down_sync(0xffffffffu, sn, o);
        ss += __shfl_down_sync(0xffffffffu, ss, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red[0][warp] = sn; red[1][warp] = ss; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a += red[0][k]; c += red[1][k]; }
        red[0][0] = a;
        red[1][0] = c;
    }
    __syncthreads();
    cplx<T>* rowN = Y + (int64_t)b * Q * (p + 1);
    cplx<T>* rowS = rowN + (int64_t)(Q - 1) * (p + 1);
    for (int m = threadIdx.x; m <= p; m += blockDim.x) {
        rowN[m] = mk<T>(m == 0 ? (T)red[0][0] : T(0), T(0));
        rowS[m] = mk<T>(m == 0 ? (T)red[1][0] : T(0), T(0));
    }
}

template <class T>
void launch_ring_fft(const hpx_plan_s* P, const T* maps, cudaStream_t s, T ew, int minN) {
    const auto& g = P->g;
    const auto& t = P->t;
    auto launch = [&](int N, int nrings, const int* list) {
        // E elements per thread: blocks of N / E threads (at least one warp)
        const bool big = N > 16 * kRingThreads;
        const int threads = std::max(32, N / (big ? 32 : 16));
        const size_t smem = (size_t)(N + N / 16) * sizeof(cplx<T>);
        auto kern = big ? ring_fft_kernel<T, 32> : ring_fft_kernel<T, 16>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dim3 grid(g.B, nrings);
        kern<<<grid, threads, smem, s>>>(
            maps, (cplx<T>*)P->Y, t.nphi, t.startN, t.startS, t.pow2, t.logn, t.fftL, t.logL, t.shOff,
            t.chOff, t.bhOff, (const cplx<T>*)t.shift, (const cplx<T>*)t.chirp, (const cplx<T>*)t.bhat,
            (const cplx<T>*)t.twid, g.Lmax, g.p, g.Q, g.npix, g.npairs, list, ew, t.shifted, g.L, P->mapIdx);
    };
    if (!P->ringList) {   // one launch sized for the largest transform
        launch(g.smem_ring, g.npairs, nullptr);
        return;
    }
    // one launch per transform length (and kind, from 4096 points up), blocks
    // sized to it, longest first
    for (const auto& c : P->ringClasses) {
        if (c.N < minN) continue;
        if (c.N < kRingCtMin) {
            launch(c.N, c.count, P->ringList + c.first);
            continue;
        }
        const size_t smem = (size_t)(c.N + c.N / 16) * sizeof(cplx<T>);
        dim3 grid(g.B, c.count);
        auto run = [&](auto kern, int threads) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kern<<<grid, threads, smem, s>>>(maps, (cplx<T>*)P->Y, t.nphi, t.startN, t.startS, t.shOff, t.chOff,
                                             t.bhOff, (const cplx<T>*)t.shift, (const cplx<T>*)t.chirp,
                                             (const cplx<T>*)t.bhat, (const cplx<T>*)t.twid, g.Lmax, g.p, g.Q,
                                             g.npix, P->ringList + c.first, ew, t.shifted, g.L, P->mapIdx);
        };
        if (c.blue && P->ringForm == 1) {   // four quarter-length Bluestein transforms, N / 16 threads
            auto run4 = [&](auto kern, int threads) {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                kern<<<grid, threads, smem, s>>>(maps, (cplx<T>*)P->Y, t.nphi, t.startN, t.startS, t.shOff,
                                                 t.ch4Off, t.bh4Off, (const cplx<T>*)t.shift,
                                                 (const cplx<T>*)t.chirp4, (const cplx<T>*)t.bhat4,
                                                 (const cplx<T>*)t.twid, g.Lmax, g.p, g.Q, g.npix,
                                                 P->ringList + c.first, ew, t.shifted, g.L, P->mapIdx);
            };
            if (c.N == 4096) run4(ring4_ct_kernel<T, 12, 256>, 256);
            else if (c.N == 8192) run4(ring4_ct_kernel<T, 13, 512>, 512);
            else run4(ring4_ct_kernel<T, 14, 512>, 512);
            continue;
        }
        // elements per thread: 16 (N / 16 threads) or, when the plan's tuning chose
        // it, 32 (N / 32 threads, two groups per thread and pass)
        const bool e32 = P->ringE == 32;
        if (c.N == 4096) {
            if (e32) { if (c.blue) run(ring_ct_kernel<T, 12, 128, true>, 128); else run(ring_ct_kernel<T, 12, 128, false>, 128); }
            else if (c.blue) run(ring_ct_kernel<T, 12, 256, true>, 256);
            else run(ring_ct_kernel<T, 12, 256, false>, 256);
        } else if (c.N == 8192) {
            if (e32) { if (c.blue) run(ring_ct_kernel<T, 13, 256, true>, 256); else run(ring_ct_kernel<T, 13, 256, false>, 256); }
            else if (c.blue) run(ring_ct_kernel<T, 13, 512, true>, 512);
            else run(ring_ct_kernel<T, 13, 512, false>, 512);
        } else {
            if (c.blue) run(ring_ct_kernel<T, 14, 512, true>, 512);
            else run(ring_ct_kernel<T, 14, 512, false>, 512);
        }
    }
}

template <class T>
void launch_poles(const hpx_plan_s* P, const T* maps, cudaStream_t s) {
    const auto& g = P->g;
    pole_kernel<T><<<g.B, 128, 0, s>>>(maps, (cplx<T>*)P->Y, P->t.poleN, P->t.poleS, P->t.polew,
                                       P->t.npole, g.p, g.Q, g.npix, P->mapIdx);
}

template void launch_ring_fft<float>(const hpx_plan_s*, const float*, cudaStream_t, float, int);
template void launch_ring_fft<double>(const hpx_plan_s*, const double*, cudaStream_t, double, int);
template void launch_poles<float>(const hpx_plan_s*, const float*, cudaStream_t);
template void launch_poles<double>(const hpx_plan_s*, const double*, cudaStream_t);

}  // namespace hpx
