// Shared-memory Stockham FFT whose length is a compile-time constant.
//
// The same algorithm as block_fft_pad_io in common.cuh (radix-16 register
// passes over a padded shared array, one spare slot every 16 elements), but
// with N, the thread count and every pass's span fixed at compile time: the
// index arithmetic of a pass reduces to one padded base per group plus
// constant offsets (folded into the shared-memory instructions), and the loops
// over groups and radix elements unroll completely.  Used where one launch
// runs many transforms of one length (the ring FFTs of step 1).
#pragma once
#include "common.cuh"

namespace hpx {
namespace ct {

__device__ __forceinline__ int padc(int i) { return i + (i >> 4); }

// cos / sin of 2 pi k / R for the odd radices 3, 5, 7 (k < R)
template <int R>
__device__ __forceinline__ double cos_r(int k) {
    if (R == 3) { constexpr double c[3] = {1.0, -0.5, -0.5}; return c[k]; }
    if (R == 5) {
        constexpr double c[5] = {1.0, 0.30901699437494742, -0.80901699437494742, -0.80901699437494742,
                                 0.30901699437494742};
        return c[k];
    }
    constexpr double c[7] = {1.0, 0.62348980185873353, -0.22252093395631440, -0.90096886790241913,
                             -0.90096886790241913, -0.22252093395631440, 0.62348980185873353};
    return c[k];
}
template <int R>
__device__ __forceinline__ double sin_r(int k) {
    if (R == 3) { constexpr double c[3] = {0.0, 0.86602540378443865, -0.86602540378443865}; return c[k]; }
    if (R == 5) {
        constexpr double c[5] = {0.0, 0.95105651629515357, 0.58778525229247313, -0.58778525229247313,
                                 -0.95105651629515357};
        return c[k];
    }
    constexpr double c[7] = {0.0, 0.78183148246802981, 0.97492791218182361, 0.43388373911755812,
                             -0.43388373911755812, -0.97492791218182361, -0.78183148246802981};
    return c[k];
}

// In-register DFT of odd prime length R (3, 5, 7): the pairs r, R - r share
// their cosines, X_q = A_q -+ i B_q, X_{R-q} = A_q +- i B_q with
// A_q = x_0 + sum_r (x_r + x_{R-r}) cos(2 pi r q / R),
// B_q = sum_r (x_r - x_{R-r}) sin(2 pi r q / R), r, q = 1 .. (R-1)/2.
template <class T, int R, bool INV>
__device__ __forceinline__ void odd_dft(cplx<T>* x) {
    constexpr int H = (R - 1) / 2;
    cplx<T> sp[H], sm[H];
    cplx<T> x0 = x[0], tot = x[0];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
        sp[r - 1] = add(x[r], x[R - r]);
        sm[r - 1] = sub(x[r], x[R - r]);
        tot = add(tot, sp[r - 1]);
    }
    cplx<T> y[R];
    y[0] = tot;
#pragma unroll
    for (int q = 1; q <= H; ++q) {
        cplx<T> A = x0, B = mk<T>(T(0), T(0));
#pragma unroll
        for (int r = 1; r <= H; ++r) {
            const int k = (r * q) % R;
            const T c = (T)cos_r<R>(k), sn = (T)sin_r<R>(k);
            A = mk<T>(A.r + c * sp[r - 1].r, A.i + c * sp[r - 1].i);
            B = mk<T>(B.r + sn * sm[r - 1].r, B.i + sn * sm[r - 1].i);
        }
        // -i B = (B.i, -B.r)
        const cplx<T> miB = mk<T>(B.i, -B.r);
        y[q] = INV ? sub(A, miB) : add(A, miB);
        y[R - q] = INV ? add(A, miB) : sub(A, miB);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = y[q];
}

// x[r] *= w^(r j) for the odd radices, each power read from the table
// (tw[t] = e^{-2 pi i t / twlen}; conjugated for INV).
template <class T, int R, bool INV>
__device__ __forceinline__ void twiddle_odd(cplx<T>* x, int j, int step, const cplx<T>* __restrict__ tw) {
#pragma unroll
    for (int r = 1; r < R; ++r) {
        cplx<T> w = tw[r * j * step];
        if (INV) w.i = -w.i;
        x[r] = mul(x[r], w);
    }
}

// One pass of radix R and span S = 2^LOGS over N elements by NT threads.
// Group k (k < N/R) takes the elements k + r N/R, multiplies element r by
// w^(r j) (w = e^{-2 pi i/(S R)}, j = k mod S), applies an R-point DFT and hands
// output q to position g S R + j + q S (g = k / S).
// LD(nat, padded) -> value and ST(nat, padded, value): element access; for the
// in-place shared-memory passes they read / write a[padded].  BAR: a barrier
// between the loads and the stores (the pass reads and writes the same array).
// tw: e^{-2 pi i t / twlen}, twstep = twlen / N.
template <class T, int N, int R, int LOGS, int NT, bool INV, bool BAR, class LD, class ST>
__device__ __forceinline__ void pass(const cplx<T>* __restrict__ tw, int twstep, LD ld, ST st) {
    constexpr int S = 1 << LOGS;
    constexpr int NG = N / R;
    constexpr int G = (NG + NT - 1) / NT;
    constexpr int IN_STRIDE = NG + NG / 16;                 // padded distance of the R inputs (NG % 16 == 0)
    static_assert(NG % 16 == 0, "pass: N / R must be a multiple of 16");
    constexpr bool ODD = (R & 1) != 0;
    const int tid = threadIdx.x;
    cplx<T> x[G][R];
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
        const int k = tid + gg * NT;
        if (NG % NT == 0 || k < NG) {
            const int pk = padc(k);
#pragma unroll
            for (int r = 0; r < R; ++r) x[gg][r] = ld(k + r * NG, pk + r * IN_STRIDE);
        }
    }
    if (BAR) __syncthreads();
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
        const int k = tid + gg * NT;
        if (NG % NT == 0 || k < NG) {
            const int j = k & (S - 1);
            if constexpr (ODD) {
                if (S > 1) twiddle_odd<T, R, INV>(x[gg], j, twstep * (N / (S * R)), tw);
                odd_dft<T, R, INV>(x[gg]);
            } else {
                if (S > 1) twiddle<T, R, INV>(x[gg], j, twstep * (N / (S * R)), tw);
                reg_dft<T, R, INV>(x[gg]);
            }
            if constexpr (S == 1) {
                static_assert(R == 16, "pass: the span-1 pass is radix 16");
#pragma unroll
                for (int q = 0; q < R; ++q) st(k * R + q, 17 * k + q, x[gg][q]);
            } else {
                static_assert(S % 16 == 0, "pass: spans above 1 are multiples of 16");
                const int base = (k >> LOGS) * S * R + j;
                const int pb = padc(base);
#pragma unroll
                for (int q = 0; q < R; ++q) st(base + q * S, pb + q * (S + S / 16), x[gg][q]);
            }
        }
    }
}

// The odd factor R0 (1, 3, 5 or 7) and log2 of the power-of-two part of a
// transform length N = R0 2^K.
template <int N>
struct Len {
    static constexpr int R0 = (N % 3 == 0) ? 3 : (N % 5 == 0) ? 5 : (N % 7 == 0) ? 7 : 1;
    static constexpr int P = N / R0;
    static constexpr int K = (P >= 2 ? 1 : 0) + (P >= 4 ? 1 : 0) + (P >= 8 ? 1 : 0) + (P >= 16 ? 1 : 0) +
                             (P >= 32 ? 1 : 0) + (P >= 64 ? 1 : 0) + (P >= 128 ? 1 : 0) + (P >= 256 ? 1 : 0) +
                             (P >= 512 ? 1 : 0) + (P >= 1024 ? 1 : 0) + (P >= 2048 ? 1 : 0) +
                             (P >= 4096 ? 1 : 0) + (P >= 8192 ? 1 : 0) + (P >= 16384 ? 1 : 0);
    static_assert((1 << K) == P, "transform length must be R0 * 2^K");
};

// Passes from span 2^LOGS (LOGS >= 4) to the last one, over the padded array a:
// radix 16 while more than 16 of the power-of-two part is left (or exactly 16
// with an odd factor still to apply), then the remaining power of two, then the
// odd radix R0 (span N / R0); the last pass hands its outputs to last_st.
template <class T, int N, int LOGS, int NT, bool INV, class ST>
__device__ __forceinline__ void rest(cplx<T>* a, const cplx<T>* __restrict__ tw, int twstep, ST last_st) {
    constexpr int R0 = Len<N>::R0;
    constexpr int LEFT = Len<N>::K - LOGS;   // log2 of the power-of-two radices still to apply
    auto lds = [&](int, int pi) { return a[pi]; };
    auto sts = [&](int, int pi, cplx<T> v) { a[pi] = v; };
    if constexpr (LEFT > 4 || (LEFT == 4 && R0 > 1)) {
        pass<T, N, 16, LOGS, NT, INV, true>(tw, twstep, lds, sts);
        __syncthreads();
        rest<T, N, LOGS + 4, NT, INV>(a, tw, twstep, last_st);
    } else if constexpr (LEFT > 0 && R0 > 1) {
        pass<T, N, (1 << LEFT), LOGS, NT, INV, true>(tw, twstep, lds, sts);
        __syncthreads();
        pass<T, N, R0, LOGS + LEFT, NT, INV, true>(tw, twstep, lds, last_st);
    } else if constexpr (LEFT > 0) {
        pass<T, N, (1 << LEFT), LOGS, NT, INV, true>(tw, twstep, lds, last_st);
    } else {
        pass<T, N, R0, LOGS, NT, INV, true>(tw, twstep, lds, last_st);
    }
}

// DFT of length N = R0 2^K (R0 in {1, 3, 5, 7}, 2^K >= 256) by NT threads: the
// first pass (radix 16) reads its inputs through ld(nat, padded) (SYNC: ld
// reads a itself, so all threads load before any stores), the passes in
// between run in the padded shared array a, and the last pass hands every
// output to st(nat, padded, value).  tw[t] = e^{-2 pi i t / twlen}, twstep =
// twlen / N.  Ends with a barrier.
template <class T, int N, int NT, bool INV, bool SYNC, class LD, class ST>
__device__ __forceinline__ void fft_n(cplx<T>* a, const cplx<T>* __restrict__ tw, int twstep, LD ld, ST st) {
    static_assert(Len<N>::K >= 8, "fft: a power-of-two part of at least 256 points");
    auto sts = [&](int, int pi, cplx<T> v) { a[pi] = v; };
    pass<T, N, 16, 0, NT, INV, SYNC>(tw, twstep, ld, sts);
    __syncthreads();
    rest<T, N, 4, NT, INV>(a, tw, twstep, st);
    __syncthreads();
}

// The same for N = 2^LOGN.
template <class T, int LOGN, int NT, bool INV, bool SYNC, class LD, class ST>
__device__ __forceinline__ void fft(cplx<T>* a, const cplx<T>* __restrict__ tw, int twstep, LD ld, ST st) {
    fft_n<T, (1 << LOGN), NT, INV, SYNC>(a, tw, twstep, ld, st);
}

}  // namespace ct
}  // namespace hpx
