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

// The same pass for a whole warp whose lanes each own one column (live = the
// lane has a column; every lane must call it, with the same n, A and coff),
// with its memory traffic taken off the critical path: the skewed angle row
// (32 complex, the same for all lanes) and each lane's input element of time
// step t are brought into a per-warp ring of RB shared-memory slots by 8-byte
// cp.async copies RB - 1 steps ahead of their use, so a step waits only for
// shared-memory loads.  ring: RB x 64 complex of this warp's shared memory.
// One Givens rotation of (carry, x) in FP32 with fixed roundings (no
// compiler-chosen contraction), so that every form of the staged sweeps gives
// the same bits: c carry + s x and c x - s carry.
__device__ __forceinline__ float rot_hi(float c, float s, float carry, float x) {
    return __fmaf_rn(c, carry, __fmul_rn(s, x));
}
__device__ __forceinline__ float rot_lo(float c, float s, float carry, float x) {
    return __fmaf_rn(c, x, -__fmul_rn(s, carry));
}

template <int RB>
struct SweepRing {
    static constexpr int kSlot = 64;   // complex per slot: 32 angles + 32 lane inputs
};

template <class T, int K, int RB>
__device__ __forceinline__ void sweep_pass_staged(cplx<T>* chain, int64_t ldc, int n, bool live,
                                                  const cplx<T>* __restrict__ A, int coff, cplx<T>* ring) {
    static_assert(sizeof(T) == 4, "staged sweeps: FP32 (8-byte complex copies)");
    constexpr int SL = SweepRing<RB>::kSlot;
    const int lane = threadIdx.x & 31;
    cplx<T> carry[K], pipe[K];
#pragma unroll
    for (int k = 0; k < K; ++k) { carry[k] = mk<T>(T(0), T(0)); pipe[k] = carry[k]; }
    const int steps = n + 2 * (K - 1);
    const int nout = n - K;   // outputs of the last stage
    auto issue = [&](int t) {
        if (t < steps) {
            cplx<T>* slot = ring + (t % RB) * SL;
            cp_async8(slot + lane, A + (int64_t)t * 32 + lane, 8);
            const bool have = live && t < n;
            cp_async8(slot + 32 + lane, have ? chain + (int64_t)t * ldc : A, have ? 8 : 0);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
#pragma unroll
    for (int q = 0; q < RB - 1; ++q) issue(q);
    for (int t = 0; t < steps; ++t) {
        __syncwarp();                 // every lane is done with the slot refilled next
        issue(t + RB - 1);
        asm volatile("cp.async.wait_group %0;" ::"n"(RB - 1) : "memory");
        __syncwarp();                 // step t's copies of all lanes are visible
        const cplx<T>* slot = ring + (t % RB) * SL;
        const cplx<T> x0 = slot[32 + lane];
        const cplx<T>* row = slot + coff;
#pragma unroll
        for (int k = K - 1; k >= 0; --k) {
            const cplx<T> x = (k == 0) ? x0 : pipe[k - 1];
            const cplx<T> cs = row[k];
            // each part rotated with the roundings of sweep_pass_staged_real
            pipe[k] = mk<T>(rot_hi(cs.r, cs.i, carry[k].r, x.r), rot_hi(cs.r, cs.i, carry[k].i, x.i));
            carry[k] = mk<T>(rot_lo(cs.r, cs.i, carry[k].r, x.r), rot_lo(cs.r, cs.i, carry[k].i, x.i));
        }
        const int j = t - 2 * K + 1;
        if (live && j >= 0 && j < nout) chain[(int64_t)j * ldc] = pipe[K - 1];
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
}

// The same pass with one real column per lane (the real or the imaginary part of
// one map's chain: the two parts share every rotation): half the registers and
// half the arithmetic of a complex lane, so batches of fewer than 32 maps fill
// twice as many lanes.  The ring slot holds the 32 angles and the 32 lanes'
// inputs (4-byte copies).
template <int K, int RB>
__device__ __forceinline__ void sweep_pass_staged_real(float* chain, int64_t ldc, int n, bool live,
                                                       const cplx<float>* __restrict__ A, int coff,
                                                       cplx<float>* ring) {
    constexpr int SL = SweepRing<RB>::kSlot;
    const int lane = threadIdx.x & 31;
    float carry[K], pipe[K];
#pragma unroll
    for (int k = 0; k < K; ++k) { carry[k] = 0.f; pipe[k] = 0.f; }
    const int steps = n + 2 * (K - 1);
    const int nout = n - K;   // outputs of the last stage
    auto issue = [&](int t) {
        if (t < steps) {
            cplx<float>* slot = ring + (t % RB) * SL;
            cp_async8(slot + lane, A + (int64_t)t * 32 + lane, 8);
            const bool have = live && t < n;
            cp_async4(reinterpret_cast<float*>(slot + 32) + lane, have ? chain + (int64_t)t * ldc : (const float*)A,
                      have ? 4 : 0);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
#pragma unroll
    for (int q = 0; q < RB - 1; ++q) issue(q);
    for (int t = 0; t < steps; ++t) {
        __syncwarp();                 // every lane is done with the slot refilled next
        issue(t + RB - 1);
        asm volatile("cp.async.wait_group %0;" ::"n"(RB - 1) : "memory");
        __syncwarp();                 // step t's copies of all lanes are visible
        const cplx<float>* slot = ring + (t % RB) * SL;
        const float x0 = reinterpret_cast<const float*>(slot + 32)[lane];
        const cplx<float>* row = slot + coff;
#pragma unroll
        for (int k = K - 1; k >= 0; --k) {
            const float x = (k == 0) ? x0 : pipe[k - 1];
            const cplx<float> cs = row[k];
            pipe[k] = rot_hi(cs.r, cs.i, carry[k], x);
            carry[k] = rot_lo(cs.r, cs.i, carry[k], x);
        }
        const int j = t - 2 * K + 1;
        if (live && j >= 0 && j < nout) chain[(int64_t)j * ldc] = pipe[K - 1];
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
}

}  // namespace hpx
