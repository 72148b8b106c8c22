// One pass of K Givens sweeps as a register wavefront (see k_rot.cu for the
// algorithm); shared by the run-time sweep kernel and the plan-time builder of
// the per-order operators.
#pragma once
#include "common.cuh"

namespace hpx {

// Angles of stages k and k+1 of one skewed row (adjacent pairs; 16-byte
// aligned for even k, which holds for every pass of two or more stages).
template <class T>
__device__ __forceinline__ void load2(const cplx<T>* p, cplx<T>& a, cplx<T>& b) {
    if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        a = mk<T>(v.x, v.y);
        b = mk<T>(v.z, v.w);
    } else {
        a = p[0];
        b = p[1];
    }
}

// One pass of K sweeps over a chain of `n` complex elements chain[i * ldc]
// (the real and imaginary parts share each rotation).  `A` points at row 0 of
// the skewed block, `coff` is the column of stage 0.
template <class T, int K>
__device__ __forceinline__ void sweep_pass(cplx<T>* chain, int64_t ldc, int n, const cplx<T>* __restrict__ A,
                                           int coff) {
    cplx<T> carry[K], pipe[K];
#pragma unroll
    for (int k = 0; k < K; ++k) { carry[k] = mk<T>(T(0), T(0)); pipe[k] = carry[k]; }
    const int steps = n + 2 * (K - 1);
    const int nout = n - K;   // outputs of the last stage
    for (int t = 0; t < steps; ++t) {
        const cplx<T> x0 = (t < n) ? chain[(int64_t)t * ldc] : mk<T>(T(0), T(0));
        const cplx<T>* row = A + (int64_t)t * 32 + coff;
        cplx<T> cs[K];
        if constexpr (K == 1) {
            cs[0] = row[0];
        } else {
#pragma unroll
            for (int k = 0; k < K; k += 2) load2(row + k, cs[k], cs[k + 1]);
        }
#pragma unroll
        for (int k = K - 1; k >= 0; --k) {
            const cplx<T> x = (k == 0) ? x0 : pipe[k - 1];
            const T c = cs[k].r, s = cs[k].i;
            pipe[k] = mk<T>(c * carry[k].r + s * x.r, c * carry[k].i + s * x.i);
            carry[k] = mk<T>(c * x.r - s * carry[k].r, c * x.i - s * carry[k].i);
        }
        const int j = t - 2 * K + 1;
        if (j >= 0 && j < nout) chain[(int64_t)j * ldc] = pipe[K - 1];
    }
}

}  // namespace hpx
