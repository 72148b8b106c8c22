// Device-side helpers shared by the HP2SPH kernels: a complex type, and an
// in-place radix-2 FFT over shared memory executed by a whole thread block.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace hpx {

template <class T>
struct __align__(2 * sizeof(T)) cplx {
    T r, i;
};

template <class T> __device__ __forceinline__ cplx<T> mk(T r, T i) { cplx<T> c; c.r = r; c.i = i; return c; }
template <class T> __device__ __forceinline__ cplx<T> add(cplx<T> a, cplx<T> b) { return mk<T>(a.r + b.r, a.i + b.i); }
template <class T> __device__ __forceinline__ cplx<T> sub(cplx<T> a, cplx<T> b) { return mk<T>(a.r - b.r, a.i - b.i); }
template <class T> __device__ __forceinline__ cplx<T> mul(cplx<T> a, cplx<T> b) {
    return mk<T>(a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r);
}
template <class T> __device__ __forceinline__ cplx<T> conjg(cplx<T> a) { return mk<T>(a.r, -a.i); }
template <class T> __device__ __forceinline__ cplx<T> scale(cplx<T> a, T s) { return mk<T>(a.r * s, a.i * s); }

// 8-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros.
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}

// 4-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros.
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}

// The power of two 2^(target - floor(log2 mx)) (clamped to normal floats), which
// brings a largest magnitude mx into [2^target, 2^(target+1)); 1 when mx is zero
// or not finite.
__device__ __forceinline__ float pow2_scale(float mx, int target) {
    if (!(mx > 0.f) || !(mx <= 3.4e38f)) return 1.f;
    const int k = max(-126, min(127, target - ilogbf(mx)));
    return __int_as_float((k + 127) << 23);
}

// Forward (sign -1) or inverse (sign +1, unnormalised) DFT of length n = 2^logn,
// in place in shared memory, by all threads of the block.  `tw` holds
// e^{-2 pi i k / twlen} for k < twlen/2 (twlen a power of two >= n).
// Decimation in time after a bit-reversal permutation.  Ends with a barrier.
template <class T>
__device__ void block_fft(cplx<T>* a, int n, int logn, const cplx<T>* __restrict__ tw, int twlen,
                          bool inverse) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < n; i += nt) {
        const int j = (int)(__brev((unsigned)i) >> (32 - logn));
        if (i < j) {
            cplx<T> t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
    __syncthreads();
    int s = 1;
    if (logn & 1) {   // one radix-2 stage so that the rest pair up
        for (int k = tid; k < (n >> 1); k += nt) {
            const cplx<T> u = a[2 * k], v = a[2 * k + 1];
            a[2 * k] = add(u, v);
            a[2 * k + 1] = sub(u, v);
        }
        __syncthreads();
        s = 2;
    }
    // two radix-2 stages (s, s+1) per pass, on the 4 elements j, j+h, j+2h, j+3h
    // of each group of 4h (h = 2^(s-1)), held in registers
    for (; s < logn; s += 2) {
        const int h = 1 << (s - 1);
        const int st1 = twlen >> s;        // e^{-2 pi i j / 2h} = tw[j * twlen / 2h]
        const int st2 = twlen >> (s + 1);  // e^{-2 pi i j / 4h}
        for (int k = tid; k < (n >> 2); k += nt) {
            const int j = k & (h - 1);
            const int i0 = ((k >> (s - 1)) << (s + 1)) + j;
            cplx<T> w1 = tw[j * st1], w2 = tw[j * st2], w3 = tw[(j + h) * st2];
            if (inverse) { w1.i = -w1.i; w2.i = -w2.i; w3.i = -w3.i; }
            const cplx<T> x0 = a[i0], x1 = a[i0 + h], x2 = a[i0 + 2 * h], x3 = a[i0 + 3 * h];
            const cplx<T> t1 = mul(x1, w1), t3 = mul(x3, w1);
            const cplx<T> y0 = add(x0, t1), y1 = sub(x0, t1), y2 = add(x2, t3), y3 = sub(x2, t3);
            const cplx<T> u2 = mul(y2, w2), u3 = mul(y3, w3);
            a[i0] = add(y0, u2);
            a[i0 + 2 * h] = sub(y0, u2);
            a[i0 + h] = add(y1, u3);
            a[i0 + 3 * h] = sub(y1, u3);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Stockham FFT over shared memory with register radix-R passes.
//
// Element i of a transform lives at a[pad(i)]: one spare slot every 16
// elements, so that the strided accesses of the passes are free of bank
// conflicts.  A pass of radix R over span S (the product of the radices done so
// far) takes, for each group k = g S + j, the R elements k + r N/R, multiplies
// element r by w^(r j) (w = e^{-2 pi i / (S R)}), applies an R-point DFT in
// registers and stores output q at g S R + j + q S.  Every thread reads all of
// its groups before a barrier and writes after it, so the pass runs in place.
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

// cos / sin of 2 pi k / 16, k = 0..7
__device__ __forceinline__ float c16f(int k) {
    constexpr float c[8] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                            0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f};
    return c[k];
}
__device__ __forceinline__ float s16f(int k) {
    constexpr float s[8] = {0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f,
                            1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f};
    return s[k];
}
__device__ __forceinline__ double c16d(int k) {
    constexpr double c[8] = {1.0, 0.92387953251128674, 0.70710678118654752, 0.38268343236508977,
                             0.0, -0.38268343236508977, -0.70710678118654752, -0.92387953251128674};
    return c[k];
}
__device__ __forceinline__ double s16d(int k) {
    constexpr double s[8] = {0.0, 0.38268343236508977, 0.70710678118654752, 0.92387953251128674,
                             1.0, 0.92387953251128674, 0.70710678118654752, 0.38268343236508977};
    return s[k];
}

// In-register R-point DFT (R = 2, 4, 8, 16): radix-2 decimation in frequency,
// then the bit-reversed outputs are renamed into natural order.
template <class T, int R, bool INV>
__device__ __forceinline__ void reg_dft(cplx<T>* x) {
#pragma unroll
    for (int half = R / 2; half >= 1; half >>= 1) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if ((i & half) == 0) {
                const int pos = i & (half - 1);
                const int k16 = pos * (8 / half);   // e^{-2 pi i pos / (2 half)} = e^{-2 pi i k16 / 16}
                const cplx<T> u = x[i], v = x[i + half];
                x[i] = add(u, v);
                const cplx<T> d = sub(u, v);
                if (pos == 0) {
                    x[i + half] = d;
                } else if (k16 == 4) {   // w = -i (forward) or +i (inverse)
                    x[i + half] = INV ? mk<T>(-d.i, d.r) : mk<T>(d.i, -d.r);
                } else if (k16 == 2 || k16 == 6) {   // w = (+-1 -+ i) / sqrt 2
                    const T h = sizeof(T) == 4 ? (T)c16f(2) : (T)c16d(2);
                    const T pr = d.r + d.i, mr = d.r - d.i;
                    if (k16 == 2) x[i + half] = INV ? mk<T>(h * mr, h * pr) : mk<T>(h * pr, -h * mr);
                    else x[i + half] = INV ? mk<T>(-h * pr, h * mr) : mk<T>(-h * mr, -h * pr);
                } else {
                    const T c = sizeof(T) == 4 ? (T)c16f(k16) : (T)c16d(k16);
                    const T s = sizeof(T) == 4 ? (T)s16f(k16) : (T)s16d(k16);
                    const T sn = INV ? s : -s;   // w = c + i sn
                    x[i + half] = mk<T>(d.r * c - d.i * sn, d.r * sn + d.i * c);
                }
            }
        }
    }
    constexpr int br2[2] = {0, 1};
    constexpr int br4[4] = {0, 2, 1, 3};
    constexpr int br8[8] = {0, 4, 2, 6, 1, 5, 3, 7};
    constexpr int br16[16] = {0, 8, 4, 12, 2, 10, 6, 14, 1, 9, 5, 13, 3, 11, 7, 15};
    cplx<T> y[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int rq = R == 16 ? br16[q] : R == 8 ? br8[q] : R == 4 ? br4[q] : br2[q];
        y[q] = x[rq];
    }
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = y[q];
}

// x[r] *= w^(r j), w^(r j) = tw[r j step] (conjugated for INV): w^j, w^2j,
// w^4j, w^8j from the table; for r = 4 hi + lo the power is (w^4j)^hi (w^j)^lo,
// with w^3j and w^12j formed once (at most two products per power).
template <class T, int R, bool INV>
__device__ __forceinline__ void twiddle(cplx<T>* x, int j, int step, const cplx<T>* __restrict__ tw) {
    auto ld = [&](int r) {
        cplx<T> w = tw[r * j * step];
        if (INV) w.i = -w.i;
        return w;
    };
    const cplx<T> b1 = ld(1);
    const cplx<T> b2 = R > 2 ? ld(2) : b1;
    const cplx<T> w3 = R > 2 ? mul(b1, b2) : b1;
    const cplx<T> b4 = R > 4 ? ld(4) : b1;
    const cplx<T> b8 = R > 8 ? ld(8) : b1;
    const cplx<T> w12 = R > 8 ? mul(b4, b8) : b1;
#pragma unroll
    for (int r = 1; r < R; ++r) {
        const int hi = r >> 2, lo = r & 3;
        const cplx<T> wl = lo == 1 ? b1 : lo == 2 ? b2 : w3;
        const cplx<T> wh = hi == 1 ? b4 : hi == 2 ? b8 : w12;
        if (hi == 0) x[r] = mul(x[r], wl);
        else if (lo == 0) x[r] = mul(x[r], wh);
        else x[r] = mul(mul(x[r], wh), wl);
    }
}

template <class T, int R, int G, bool INV>
__device__ __forceinline__ void stockham_pass(cplx<T>* a, int N, int logS, const cplx<T>* __restrict__ tw,
                                              int twlen) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ngroups = N / R;
    const int S = 1 << logS;
    cplx<T> x[G][R];
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
        const int k = tid + gg * nt;
        if (k < ngroups) {
#pragma unroll
            for (int r = 0; r < R; ++r) x[gg][r] = a[pad(k + r * ngroups)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
        const int k = tid + gg * nt;
        if (k < ngroups) {
            const int j = k & (S - 1);
            const int g = k >> logS;
            if (S > 1) twiddle<T, R, INV>(x[gg], j, twlen / (S * R), tw);
            reg_dft<T, R, INV>(x[gg]);
            const int base = g * S * R + j;
#pragma unroll
            for (int q = 0; q < R; ++q) a[pad(base + q * S)] = x[gg][q];
        }
    }
    __syncthreads();
}

// First pass (span 1, no twiddles) with the inputs taken from ld(i), i < N,
// instead of read directly; its outputs go to the padded array a.  SYNC: ld
// reads a itself, so every thread loads before any thread stores.  Ends with a
// barrier.
template <class T, int R, int G, bool INV, bool SYNC, class LD>
__device__ __forceinline__ void stockham_first(cplx<T>* a, int N, LD ld) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ngroups = N / R;
    cplx<T> x[G][R];
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
        const int k = tid + gg * nt;
        if (k < ngroups) {
#pragma unroll
            for (int r = 0; r < R; ++r) x[gg][r] = ld(k + r * ngroups);
        }
    }
    if (SYNC) __syncthreads();
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
        const int k = tid + gg * nt;
        if (k < ngroups) {
            reg_dft<T, R, INV>(x[gg]);
#pragma unroll
            for (int q = 0; q < R; ++q) a[pad(k * R + q)] = x[gg][q];
        }
    }
    __syncthreads();
}

// Last pass (span S = N / R) in place in a, storing f(j, value) for output j
// (natural order).  Ends with a barrier.
template <class T, int R, int G, bool INV, class F>
__device__ __forceinline__ void stockham_last_f(cplx<T>* a, int N, const cplx<T>* __restrict__ tw, int twlen, F f) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int S = N / R;
    cplx<T> x[G][R];
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
        const int j = tid + gg * nt;
        if (j < S) {
#pragma unroll
            for (int r = 0; r < R; ++r) x[gg][r] = a[pad(j + r * S)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
        const int j = tid + gg * nt;
        if (j < S) {
            twiddle<T, R, INV>(x[gg], j, twlen / N, tw);
            reg_dft<T, R, INV>(x[gg]);
#pragma unroll
            for (int q = 0; q < R; ++q) a[pad(j + q * S)] = f(j + q * S, x[gg][q]);
        }
    }
    __syncthreads();
}

// DFT of length N = 2^logn (5 <= logn, N <= E * blockDim; forward, or inverse
// unnormalised) in the padded shared array a, whose input element i is ld(i)
// (SYNC: ld reads a) and whose output element j is stored as f(j, value).
template <class T, int E, bool INV, bool SYNC, class LD, class F>
__device__ __forceinline__ void block_fft_pad_io(cplx<T>* a, int logn, const cplx<T>* __restrict__ tw, int twlen,
                                                 LD ld, F f) {
    const int N = 1 << logn;
    stockham_first<T, 16, E / 16, INV, SYNC>(a, N, ld);
    int logS = 4;
    const int lr = logn & 3;
    const int last = lr == 0 ? logn - 4 : logn - lr;
    for (; logS < last; logS += 4) stockham_pass<T, 16, E / 16, INV>(a, N, logS, tw, twlen);
    if (lr == 0) stockham_last_f<T, 16, E / 16, INV>(a, N, tw, twlen, f);
    else if (lr == 3) stockham_last_f<T, 8, E / 8, INV>(a, N, tw, twlen, f);
    else if (lr == 2) stockham_last_f<T, 4, E / 4, INV>(a, N, tw, twlen, f);
    else stockham_last_f<T, 2, E / 2, INV>(a, N, tw, twlen, f);
}

// Last pass (span S = N / R) reading a and handing output j (natural order,
// all j < N) to st(j, value) instead of storing it.  No barrier.
template <class T, int R, int G, class ST>
__device__ __forceinline__ void stockham_last(const cplx<T>* a, int N, const cplx<T>* __restrict__ tw, int twlen,
                                              ST st) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int S = N / R;
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
        const int j = tid + gg * nt;
        if (j < S) {
            cplx<T> x[R];
#pragma unroll
            for (int r = 0; r < R; ++r) x[r] = a[pad(j + r * S)];
            twiddle<T, R, false>(x, j, twlen / N, tw);
            reg_dft<T, R, false>(x);
#pragma unroll
            for (int q = 0; q < R; ++q) st(j + q * S, x[q]);
        }
    }
}

// Forward DFT of length N = 2^logn (5 <= logn, N <= E * blockDim) whose input
// element i is ld(i) and whose output element j is handed to st(j, value): the
// first pass reads through ld, the last pass writes through st, the passes in
// between run in the padded shared array a.
template <class T, int E, class LD, class ST>
__device__ __forceinline__ void block_fft_io(cplx<T>* a, int logn, const cplx<T>* __restrict__ tw, int twlen, LD ld,
                                             ST st) {
    const int N = 1 << logn;
    stockham_first<T, 16, E / 16, false, false>(a, N, ld);
    int logS = 4;
    const int lr = logn & 3;   // radix of the last pass: 16 if lr == 0, else 2^lr
    const int last = lr == 0 ? logn - 4 : logn - lr;   // logS of the last pass
    for (; logS < last; logS += 4) stockham_pass<T, 16, E / 16, false>(a, N, logS, tw, twlen);
    if (lr == 0) stockham_last<T, 16, E / 16>(a, N, tw, twlen, st);
    else if (lr == 3) stockham_last<T, 8, E / 8>(a, N, tw, twlen, st);
    else if (lr == 2) stockham_last<T, 4, E / 4>(a, N, tw, twlen, st);
    else stockham_last<T, 2, E / 2>(a, N, tw, twlen, st);
}

// DFT of length N = 2^logn (forward sign -1, or inverse +1 unnormalised) of the
// padded shared array a, by all threads of the block.  E = elements per thread
// and pass (16 or 32): radix-16 passes with E/16 groups per thread, then one
// pass of the remaining radix with E/R groups; the caller guarantees
// N <= E * blockDim.  `tw` holds e^{-2 pi i k / twlen} for k < twlen (the full
// circle).  Ends with a barrier.
template <class T, int E>
__device__ __forceinline__ void block_fft_pad(cplx<T>* a, int logn, const cplx<T>* __restrict__ tw, int twlen,
                                              bool inverse) {
    const int N = 1 << logn;
    int logS = 0;
    if (inverse) {
        for (; logn - logS >= 4; logS += 4) stockham_pass<T, 16, E / 16, true>(a, N, logS, tw, twlen);
        const int lr = logn - logS;
        if (lr == 3) stockham_pass<T, 8, E / 8, true>(a, N, logS, tw, twlen);
        else if (lr == 2) stockham_pass<T, 4, E / 4, true>(a, N, logS, tw, twlen);
        else if (lr == 1) stockham_pass<T, 2, E / 2, true>(a, N, logS, tw, twlen);
    } else {
        for (; logn - logS >= 4; logS += 4) stockham_pass<T, 16, E / 16, false>(a, N, logS, tw, twlen);
        const int lr = logn - logS;
        if (lr == 3) stockham_pass<T, 8, E / 8, false>(a, N, logS, tw, twlen);
        else if (lr == 2) stockham_pass<T, 4, E / 4, false>(a, N, logS, tw, twlen);
        else if (lr == 1) stockham_pass<T, 2, E / 2, false>(a, N, logS, tw, twlen);
    }
}

}  // namespace hpx
