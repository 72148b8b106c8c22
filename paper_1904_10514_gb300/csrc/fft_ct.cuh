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

// One pass of radix R and span S = 2^LOGS over N elements by NT threads.
// Group k (k < N/R) takes the elements k + r N/R, multiplies element r by
// w^(r j) (w = e^{-2 pi i/(S R)}, j = k mod S), applies an R-point DFT and hands
// output q to position g S R + j + q S (g = k / S).
// LD(nat, padded) -> value and ST(nat, padded, value): element access; for the
// in-place shared-memory passes they read / write a[padded].  BAR: a barrier
// between the loads and the stores (the pass reads and writes the same array).
// tw: e^{-2 pi i t / twlen}, twstep = twlen / N.
// tid: this thread's index among the NT threads of the transform (a block may
// run several transforms side by side, each on its own NT threads and array).
template <class T, int N, int R, int LOGS, int NT, bool INV, bool BAR, class LD, class ST>
__device__ __forceinline__ void pass(const cplx<T>* __restrict__ tw, int twstep, LD ld, ST st, int tid) {
    constexpr int S = 1 << LOGS;
    constexpr int NG = N / R;
    constexpr int G = (NG + NT - 1) / NT;
    constexpr int IN_STRIDE = NG + NG / 16;                 // padded distance of the R inputs (NG % 16 == 0)
    static_assert(NG % 16 == 0, "pass: N / R must be a multiple of 16");
    static_assert(NG % NT == 0 || G == 1, "pass: groups must split evenly over the threads");
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
            if (S > 1) twiddle<T, R, INV>(x[gg], j, twstep * (N / (S * R)), tw);
            reg_dft<T, R, INV>(x[gg]);
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

// Passes of span 16^s, s >= 1, up to the last one, over the padded array a.
template <class T, int LOGN, int LOGS, int NT, bool INV, class ST>
__device__ __forceinline__ void rest(cplx<T>* a, const cplx<T>* __restrict__ tw, int twstep, ST last_st, int tid) {
    constexpr int N = 1 << LOGN;
    constexpr int LEFT = LOGN - LOGS;   // log2 of the radices still to apply
    auto lds = [&](int, int pi) { return a[pi]; };
    auto sts = [&](int, int pi, cplx<T> v) { a[pi] = v; };
    if constexpr (LEFT > 4) {
        pass<T, N, 16, LOGS, NT, INV, true>(tw, twstep, lds, sts, tid);
        __syncthreads();
        rest<T, LOGN, LOGS + 4, NT, INV>(a, tw, twstep, last_st, tid);
    } else {
        constexpr int R = 1 << LEFT;
        pass<T, N, R, LOGS, NT, INV, true>(tw, twstep, lds, last_st, tid);
    }
}

// DFT of length N = 2^LOGN (LOGN >= 8) by NT threads: the first pass reads its
// inputs through ld(nat, padded) (SYNC: ld reads a itself, so all threads load
// before any stores), the passes in between run in the padded shared array a,
// and the last pass hands every output to st(nat, padded, value).  Ends with a
// barrier.  The barriers are the block's: side-by-side transforms (tid = the
// thread's index in its transform's group) run their passes in step.
template <class T, int LOGN, int NT, bool INV, bool SYNC, class LD, class ST>
__device__ __forceinline__ void fft(cplx<T>* a, const cplx<T>* __restrict__ tw, int twstep, LD ld, ST st,
                                    int tid = -1) {
    constexpr int N = 1 << LOGN;
    static_assert(LOGN >= 8, "fft: at least 256 points");
    if (tid < 0) tid = threadIdx.x;
    auto sts = [&](int, int pi, cplx<T> v) { a[pi] = v; };
    pass<T, N, 16, 0, NT, INV, SYNC>(tw, twstep, ld, sts, tid);
    __syncthreads();
    rest<T, LOGN, 4, NT, INV>(a, tw, twstep, st, tid);
    __syncthreads();
}

}  // namespace ct
}  // namespace hpx
