// Per-order operators on the 5th-generation tensor cores (tcgen05, TMEM).
//
// The contraction a_{m+c+2i}^m[map] = sum_k M_{m,c}[i][k] b[map][m][par][k] of
// k_fused.cu, for FP32 plans, with FP32-level accuracy from lower-precision
// tensor-core MMAs: every operand x is split into a pair hi + lo of numbers of
// 11 significant bits (|x - hi - lo| <= 2^-22 |x|) and the product is
// accumulated as
//     A_hi B_lo + A_lo B_hi + A_hi B_hi
// (the dropped A_lo B_lo term is below 2^-22 of the product).  One CTA
// computes a tile of 128 rows (degrees of one chain) x 64 real columns (real
// parts of 32 maps, then their imaginary parts) over K = P2 in chunks of 32.
// The plan stores M tile by tile as consecutive K-chunks in the MMA's K-major,
// no-swizzle core-matrix order, so a chunk is one contiguous block of rp x 128
// bytes that one bulk copy brings into shared memory.  Each chunk goes into a
// fresh TMEM accumulator whose value is added to FP32 registers: every
// tensor-core accumulation then stays at the size of one chunk's partial sum,
// and the registers add 1 + K/32 terms with round-to-nearest.
//
// Two forms (HPX_TC_F16):
//   1 (default) fused_tc_ws_kernel: hi / lo are FP16 numbers of the operands
//     after power-of-two scaling (M converted at plan time), kind::f16 MMAs,
//     warp-specialised (description below);
//   0 fused_tc_tmem_kernel: hi / lo are TF32 numbers, kind::tf32 MMAs; the
//     threads split each chunk of M into tensor memory and of b into shared
//     memory, with one block barrier per chunk.
// Every wait is bounded: on timeout the CTA records HPX_ERR_TIMEOUT in the
// plan's status word, waits (bounded) for its copies and MMAs still in flight
// and returns after releasing its tensor memory.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>

#include "fp16pair.cuh"
#include "plan.h"
#include "plan_math.h"

#ifndef HPX_TC_F16
#define HPX_TC_F16 1
#endif

namespace hpx {

namespace {

constexpr int TM = 128;          // rows per tile (MMA M)
constexpr int TN = 64;           // real columns per tile (MMA N): 32 maps x (re, im)
constexpr int KC = 32;           // K per chunk
constexpr int TILE_A = TM * KC * 4;   // bytes of one operator chunk (16 KB)
constexpr int TILE_B = TN * KC * 4;   // bytes of one TF32 copy of a b chunk (8 KB)
constexpr int NT = 256;          // threads per CTA of the TF32 form
constexpr uint32_t kSpinLimit = 1u << 26;
constexpr int NSA = 4;           // operator stages of the TF32 form

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major, no swizzle, SM100 version bits.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version
    return d;                 // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major,
// M = 128, N = 64.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

// kind::tf32 MMA with A read from tensor memory (lane = row, one 32-bit column per k).
__device__ __forceinline__ void mma_tf32_ta(uint32_t dtmem, uint32_t atmem, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n"
        :
        : "r"(dtmem), "r"(atmem), "l"(bdesc), "r"(kIdesc), "r"(acc));
}

// 16 consecutive 32-bit columns of this warp's 32 TMEM lanes (one per thread).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        :
        : "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
          "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// One-dimensional bulk copy global -> shared memory of `bytes` (a multiple of
// 16, both addresses 16-byte aligned) that completes as transaction bytes on
// the mbarrier; the source lines are marked evict-first in L2 (the operators
// are streamed once per call, the right-hand sides are reused).
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile(
        "{\n\t.reg .b64 pol;\n\t"
        "createpolicy.fractional.L2::evict_first.b64 pol, 1.0;\n\t"
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], pol;\n\t}\n"
        :
        : "r"(dst), "l"(src), "r"(bytes), "r"(mbar)
        : "memory");
}

// Arrive on the mbarrier (count 1) announcing `bytes` of transactions.
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Bounded wait for the given phase parity; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t limit = kSpinLimit) {
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// x rounded to the nearest TF32 number (10 stored mantissa bits; ties away from
// zero): add half a TF32 ulp to the magnitude bits and clear the low 13 bits.
__device__ __forceinline__ uint32_t tf32_rn(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }

// x = hi + lo + r with hi, lo TF32 numbers and |r| <= 2^-22 |x|: hi is x rounded
// to TF32, x - hi is exact in FP32 and is rounded to TF32 in turn.
struct Split {
    uint32_t hi, lo;
};
__device__ __forceinline__ Split split(float x) {
    const uint32_t h = tf32_rn(x);
    return Split{h, tf32_rn(x - __uint_as_float(h))};
}

}  // namespace

// TF32 form: the chunks of the operator tile are copied by one thread into a
// ring of NSA shared-memory stages with cp.async.bulk, NSA chunks ahead of their
// use; every thread reads the 16 consecutive k of one row of the chunk (row =
// its TMEM lane, k half = warp / 4; 8 lanes cover 128 contiguous bytes: no bank
// conflicts), splits them in registers and stores the hi and lo parts to TMEM
// with tcgen05.st; b is loaded into registers two chunks ahead and split into
// shared memory.  One thread issues 4 K-steps x 3 kind::tf32 MMAs (M = 128,
// N = 64, K = 8, A from TMEM) into a fresh accumulator and commits them to the
// stage's mbarrier; the threads then wait for the previous chunk's MMAs and add
// its accumulator (tcgen05.ld; warp w owns TMEM lanes 32 (w mod 4) .. +31).
// TMEM per CTA (256 columns): accumulators of stage s at 64 s, A hi / lo of
// stage s at 128 + 64 s and 128 + 64 s + 32.  Shared memory: [NSA operator
// stages] [two stages of (Bhi, Blo)].
__global__ void __launch_bounds__(NT, 2) fused_tc_tmem_kernel(
    const float* __restrict__ Mt, const int64_t* __restrict__ tcOff, const int* __restrict__ tiles,
    const cplx<float>* __restrict__ bvec, cplx<float>* __restrict__ alm, int P2, int p, int L, int B, int64_t nalm,
    int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_all[];
    unsigned char* const sA = smem_all;                  // NSA x TILE_A
    unsigned char* const smem = smem_all + NSA * TILE_A;   // two stages of (Bhi, Blo)
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ __align__(8) uint64_t fullA[NSA];
    __shared__ uint32_t tmem_base;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = tiles[3 * blockIdx.x], c = tiles[3 * blockIdx.x + 1], i0 = tiles[3 * blockIdx.x + 2];
    const int par = ((m & 1) + c) & 1;
    const int nrows = chain_len(m, c, L);
    const int rp = (min(TM, nrows - i0) + 7) & ~7;
    const int b0 = blockIdx.y * (TN / 2);
    const float* At = Mt + tcOff[blockIdx.x];
    const int row = 32 * (warp & 3) + lane, khalf = warp >> 2;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    const int nchunks = (P2 + KC - 1) / KC;
    const uint32_t chunkBytes = (uint32_t)rp * 128u;
    int issuedA = 0, doneA = 0;   // bulk copies issued / seen complete (thread 0)
    auto issueA = [&](int ch) {   // thread 0: chunk ch into stage ch % NSA
        const uint32_t fb = smem_u32(&fullA[ch % NSA]);
        mbar_expect_tx(fb, chunkBytes);
        bulk_g2s(smem_u32(sA + (ch % NSA) * TILE_A), At + (int64_t)ch * rp * 32, chunkBytes, fb);
        issuedA = ch + 1;
    };
    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        for (int q = 0; q < NSA; ++q) mbar_init(smem_u32(&fullA[q]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int q = 0; q < NSA && q < nchunks; ++q) issueA(q);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t dtmem = tmem_base;
    const uint32_t lanebits = (uint32_t)(32 * (warp & 3)) << 16;

    const int bl = 8 * (warp & 3) + (lane & 7);
    const int kq = 4 * (warp >> 2) + (lane >> 3);
    const int bmap = b0 + bl;
    const cplx<float>* bsrc = bvec + (((int64_t)min(bmap, B - 1) * (p + 1) + m) * 2 + par) * P2;

    float2 rbA[4], rbB[4];
    auto load_chunk = [&](int ch, float2 (&rb)[4]) {
        const int k = ch * KC + 4 * kq;
#pragma unroll
        for (int e = 0; e < 4; ++e)
            rb[e] = (bmap < B && k + e < P2) ? __ldg(reinterpret_cast<const float2*>(bsrc + k + e))
                                             : make_float2(0.f, 0.f);
    };
    auto store_chunk = [&](int ch, const float2 (&rb)[4]) {
        const int st = ch & 1;
        float4 ra[4];   // this row's 16 values of the chunk from its shared-memory stage
        {
            const unsigned char* a = sA + (ch % NSA) * TILE_A + (row >> 3) * 1024 + (row & 7) * 16;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                ra[q] = row < rp ? *reinterpret_cast<const float4*>(a + (4 * khalf + q) * 128)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        uint32_t hi[16], lo[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float v[4] = {ra[q].x, ra[q].y, ra[q].z, ra[q].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const Split sp = split(v[e]);
                hi[4 * q + e] = sp.hi;
                lo[4 * q + e] = sp.lo;
            }
        }
        const uint32_t acol = 128 + 64 * st + 16 * khalf;
        tmem_st16(dtmem + lanebits + acol, hi);
        tmem_st16(dtmem + lanebits + acol + 32, lo);
        unsigned char* Bhi = smem + st * (2 * TILE_B);
        unsigned char* Blo = Bhi + TILE_B;
        const uint32_t offr = (uint32_t)((bl >> 3) * 1024 + kq * 128 + (bl & 7) * 16);
        const uint32_t offi = offr + 4 * 1024;
        const Split r0 = split(rb[0].x), r1 = split(rb[1].x), r2 = split(rb[2].x), r3 = split(rb[3].x);
        const Split q0 = split(rb[0].y), q1 = split(rb[1].y), q2 = split(rb[2].y), q3 = split(rb[3].y);
        *reinterpret_cast<uint4*>(Bhi + offr) = make_uint4(r0.hi, r1.hi, r2.hi, r3.hi);
        *reinterpret_cast<uint4*>(Blo + offr) = make_uint4(r0.lo, r1.lo, r2.lo, r3.lo);
        *reinterpret_cast<uint4*>(Bhi + offi) = make_uint4(q0.hi, q1.hi, q2.hi, q3.hi);
        *reinterpret_cast<uint4*>(Blo + offi) = make_uint4(q0.lo, q1.lo, q2.lo, q3.lo);
    };

    float acc[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) acc[q] = 0.f;
    const uint32_t tsub = dtmem + lanebits + (uint32_t)(32 * (warp >> 2));
    auto drain = [&](int st) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t v[16];
            tmem_ld16(tsub + (uint32_t)(st * TN + 16 * h), v);
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[16 * h + q] += __uint_as_float(v[q]);
        }
    };

    bool ok = true;
    int issued = 0;
    auto step = [&](int ch, float2 (&rb)[4]) {
        const int st = ch & 1;
        // the chunk's bulk copy has landed
        if (!mbar_wait(smem_u32(&fullA[ch % NSA]), (uint32_t)((ch / NSA) & 1))) ok = false;
        else if (tid == 0) doneA = ch + 1;
        // stage st (A in TMEM, b in shared memory) was read by the MMAs of chunk
        // ch - 2, which completed before their accumulator was drained
        store_chunk(ch, rb);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (__syncthreads_or(!ok)) {
            ok = false;
            return false;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t bH = smem_u32(smem + st * (2 * TILE_B)), bL = bH + TILE_B;
            const uint32_t aH = dtmem + 128 + 64 * st, aL = aH + 32;
            const uint32_t d = dtmem + (uint32_t)(st * TN);
#pragma unroll
            for (int ks = 0; ks < KC / 8; ++ks) {
                const uint32_t o = ks * 256;
                mma_tf32_ta(d, aH + 8 * ks, make_desc(bL + o, 128, 1024), ks > 0 ? 1u : 0u);
                mma_tf32_ta(d, aL + 8 * ks, make_desc(bH + o, 128, 1024), 1u);
            }
#pragma unroll
            for (int ks = 0; ks < KC / 8; ++ks) {
                const uint32_t o = ks * 256;
                mma_tf32_ta(d, aH + 8 * ks, make_desc(bH + o, 128, 1024), 1u);
            }
            mma_commit(smem_u32(&mbar[st]));
            // every thread has read operator stage ch % NSA (before the barrier)
            if (ch + NSA < nchunks) issueA(ch + NSA);
        }
        issued = ch + 1;
        if (ch + 2 < nchunks) load_chunk(ch + 2, rb);
        if (ch > 0) {
            const int sp = st ^ 1;
            if (!mbar_wait(smem_u32(&mbar[sp]), (uint32_t)(((ch - 1) >> 1) & 1))) ok = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (ok) drain(sp);
        }
        return true;
    };
    load_chunk(0, rbA);
    if (nchunks > 1) load_chunk(1, rbB);
    for (int ch = 0; ch < nchunks; ch += 2) {
        if (!step(ch, rbA)) break;
        if (ch + 1 < nchunks && !step(ch + 1, rbB)) break;
    }
    if (ok) {
        const int cl = nchunks - 1;
        if (!mbar_wait(smem_u32(&mbar[cl & 1]), (uint32_t)((cl >> 1) & 1))) ok = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ok) drain(cl & 1);
    }
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            atomicExch(status, HPX_ERR_TIMEOUT);
            if (issued > 0) mbar_wait(smem_u32(&mbar[(issued - 1) & 1]), (uint32_t)(((issued - 1) >> 1) & 1));
            // bulk copies still in flight into this CTA's shared memory
            for (int q = doneA; q < issuedA; ++q) mbar_wait(smem_u32(&fullA[q % NSA]), (uint32_t)((q / NSA) & 1));
        }
    } else {
        const int i = i0 + 32 * (warp & 3) + lane;
        if (i < nrows) {
            const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2 + m + c + 2 * (int64_t)i;
            float* out = reinterpret_cast<float*>(alm) + 2 * base + (warp >> 2);
#pragma unroll
            for (int q = 0; q < 32; ++q)
                if (b0 + q < B) out[2 * (int64_t)(b0 + q) * nalm] = acc[q];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(dtmem), "r"(256) : "memory");
}

// ---------------------------------------------------------------- FP16 form
//
// The same contraction with every FP32 number x represented as a pair of FP16
// numbers after a power-of-two scaling: x' = s x, hi = fp16(x'), lo = fp16(x' - hi)
// (x' - hi is exact in FP32, and |x' - hi - lo| <= 2^-22 |x'| while lo is an FP16
// normal number).  Each row of M is scaled so that its largest entry lies in
// [2^14, 2^15) (plan time, tc_to_f16_kernel); each column of b (one map, one
// order: both parities, real and imaginary parts) so that its largest entry lies
// in [2^13, 2^14) (the grid-FFT kernels record its largest magnitude, bscale).  The products of
// FP16 numbers are exact in the FP32 accumulator, and
//     A_hi B_lo + A_lo B_hi + A_hi B_hi
// carries the same 2^-22 relative error per product as 3xTF32, in 3 kind::f16
// MMAs (K = 16) at twice the TF32 rate.  Entries below 2^-18 of their row (or
// column) maximum lose relative precision, with an absolute error below 2^-39
// of that maximum.  The scales are undone in the epilogue.
//
// The right-hand sides arrive already split: the grid-FFT kernel that
// produces b scales every column and writes its FP16 pairs in the MMA's B
// layout (bpk: per map tile of 32, order m, parity and K-chunk one 8 KB block,
// the hi copy then the lo copy, each 64 columns x 32 k in K-major core matrices
// of 8 columns x 8 halves: 8-column groups 512 bytes apart, core matrices
// adjacent in K 128 bytes apart; columns 0-31 the real parts of the 32 maps,
// 32-63 the imaginary parts), so the kernel converts nothing.
//
// The kernel is warp-specialised; its roles meet only at mbarriers, so each
// stream runs ahead by its own ring of stages:
//   * warp 4 (one lane) copies each K-chunk's operator block (hi then lo,
//     rp x 64 bytes each) and its 8 KB b block into one of NSH shared-memory
//     stages by two bulk copies that complete on the stage's mbarrier (fullA /
//     emptyA);
//   * warp 5 (one lane) issues, per chunk, 2 K-steps x 3 kind::f16 MMAs
//     (M = 128, N = 64, K = 16) into a fresh accumulator of NACC TMEM stages
//     (64 columns each) and commits them to emptyA and accFull;
//   * warps 0-3 (128 workers) drain each accumulator into FP32 registers
//     (thread = TMEM lane = row; 32 real and 32 imaginary columns), release it
//     (accEmpty), and write the tile's results.
// Every wait is bounded and watches an abort flag: a role that gives up sets
// it, the others stop at their next wait, and one thread then waits (bounded)
// for the bulk copies and MMAs still in flight before the CTA releases its
// tensor memory.

constexpr int TILE_H = TN * KC * 2;   // bytes of one FP16 copy of a b chunk (4 KB)
constexpr int TILE_BP = kBpkChunk;    // a b chunk's pair (hi, lo): 8 KB
static_assert(TILE_BP == 2 * TILE_H, "packed b chunk: hi and lo copies");
constexpr int NSH = 4;                // stages (operator chunk + b chunk)
constexpr int NACC = 4;               // accumulator stages (TMEM, 64 columns each)
constexpr int NW = 128;               // worker threads (warps 0-3)
constexpr int NTW = NW + 64;          // + the copy warp and the MMA warp

// Instruction descriptor: kind::f16, D = F32, A = B = F16, both K-major,
// M = 128, N = 64.
constexpr uint32_t kIdescH = (1u << 4) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(dtmem), "l"(adesc), "l"(bdesc), "r"(kIdescH), "r"(acc));
}

// Bulk copy with the default L2 policy (data that other CTAs read again).
__device__ __forceinline__ void bulk_g2s_keep(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// Bounded wait that also gives up when another role has set *abort.
__device__ __forceinline__ bool ws_wait(uint32_t mbar, uint32_t parity, volatile int* abort) {
    for (uint32_t it = 0; it < kSpinLimit; ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63) == 63 && *abort) return false;
    }
    *abort = 1;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// MODE 0: the per-order operators M_{m,c}, tile (m, c, i0), output into alm.
// MODE 1: the latitude operator D of the sweeps path (Sec. 3.2.2 and the first
// half of Sec. 3.3, shared by all orders of one parity), tile (m, par, i0) =
// rows q = i0.. of D[m & 1][par] applied to the columns b[map][m][par], output
// into beta[m][par][q][map] for the Givens sweeps; the tiles of all orders of
// one parity point at the same operator data, which stays resident in L2
// (default copy policy; the per-order operators are streamed once per call and
// copied evict-first).
// MODE 2: the synthesis' order-m conversion, the transposed contraction
// X[map][m][par][k] = sum_i S_{m,c}[i][k] a_{m+c+2i}^m[map]: tile (m, c, k0) =
// rows k = k0.. of S_{m,c}^T (P2 rows), K = the chain's degrees (its own
// chunk count), B = the packed coefficients of chain c (scaled per (map, m, c)),
// output into bvec[map][m][par][k]; 1 / row scale at rowBase[tile] + row.
template <int MODE>
__global__ void __launch_bounds__(NTW, 2) fused_tc_ws_kernel(
    const unsigned char* __restrict__ Mh, const int64_t* __restrict__ tcOff, const float* __restrict__ tcRinv,
    const int* __restrict__ tiles, const unsigned char* __restrict__ bpk, const float* __restrict__ bscale,
    cplx<float>* __restrict__ alm, int P2, int p, int L, int B, int64_t nalm, int* __restrict__ status,
    const int64_t* __restrict__ rowBase) {
    constexpr bool DENSE = MODE == 1, SYNTH = MODE == 2;
    extern __shared__ __align__(1024) unsigned char smem_w[];
    unsigned char* const sA = smem_w;                  // NSH x TILE_A: operator chunks (hi, lo)
    unsigned char* const sB = smem_w + NSH * TILE_A;   // NSH x TILE_BP: b chunks (hi, lo)
    __shared__ __align__(8) uint64_t fullA[NSH], emptyA[NSH], accFull[NACC], accEmpty[NACC];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_, issuedA, seenA, committed;
    __shared__ float tinv[TN / 2];   // 1 / column scale of each map of the tile

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = tiles[3 * blockIdx.x], c = tiles[3 * blockIdx.x + 1], i0 = tiles[3 * blockIdx.x + 2];
    const int par = DENSE ? c : ((m & 1) + c) & 1;
    const int nrows = (DENSE || SYNTH) ? P2 : chain_len(m, c, L);
    const int rp = (min(TM, nrows - i0) + 7) & ~7;
    const int b0 = blockIdx.y * (TN / 2);
    const int nchB = (P2 + KC - 1) / KC;                                       // K-chunks of a packed half
    const int nchunks = SYNTH ? (chain_len(m, c, L) + KC - 1) / KC : nchB;    // K-chunks of this tile
    const uint32_t chunkBytes = (uint32_t)rp * 128u;
    volatile int* abort = &abort_;

    if (warp == 0) {   // NACC x 64 accumulator columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(NACC * TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < NSH; ++q) {
            mbar_init(smem_u32(&fullA[q]), 1);
            mbar_init(smem_u32(&emptyA[q]), 1);
        }
        for (int q = 0; q < NACC; ++q) {
            mbar_init(smem_u32(&accFull[q]), 1);
            mbar_init(smem_u32(&accEmpty[q]), NW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_ = 0;
        issuedA = 0;
        seenA = 0;
        committed = 0;
    }
    if (tid < TN / 2) {
        const int bm = b0 + tid;
        const int64_t col = SYNTH ? ((int64_t)bm * (L + 1) + m) * 2 + c : (int64_t)bm * (L + 1) + m;
        tinv[tid] = bm < B ? 1.f / pow2_scale(bscale[col], 13) : 0.f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t dtmem = tmem_base;

    if (warp == 4) {
        // ---------------------------------------------------------- copies
        if (lane == 0) {
            const unsigned char* At = Mh + tcOff[blockIdx.x] * 4;
            const unsigned char* Bt =
                bpk + (((int64_t)blockIdx.y * (L + 1) + m) * 2 + (SYNTH ? c : par)) * nchB * TILE_BP;
            for (int ch = 0; ch < nchunks; ++ch) {
                const int s = ch % NSH;
                if (ch >= NSH && !ws_wait(smem_u32(&emptyA[s]), (uint32_t)((ch / NSH + 1) & 1), abort)) break;
                const uint32_t fb = smem_u32(&fullA[s]);
                mbar_expect_tx(fb, chunkBytes + TILE_BP);
                if (DENSE) bulk_g2s_keep(smem_u32(sA + s * TILE_A), At + (int64_t)ch * chunkBytes, chunkBytes, fb);
                else bulk_g2s(smem_u32(sA + s * TILE_A), At + (int64_t)ch * chunkBytes, chunkBytes, fb);
                bulk_g2s_keep(smem_u32(sB + s * TILE_BP), Bt + (int64_t)ch * TILE_BP, TILE_BP, fb);
                issuedA = ch + 1;
            }
        }
    } else if (warp == 5) {
        // ---------------------------------------------------------- MMAs
        if (lane == 0) {
            for (int ch = 0; ch < nchunks; ++ch) {
                const int s = ch % NSH, a = ch % NACC;
                if (!ws_wait(smem_u32(&fullA[s]), (uint32_t)((ch / NSH) & 1), abort)) break;
                seenA = ch + 1;
                if (ch >= NACC && !ws_wait(smem_u32(&accEmpty[a]), (uint32_t)((ch / NACC + 1) & 1), abort)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t aH = smem_u32(sA + s * TILE_A), aL = aH + (uint32_t)rp * 64;
                const uint32_t bH = smem_u32(sB + s * TILE_BP), bL = bH + TILE_H;
                const uint32_t d = dtmem + (uint32_t)(a * TN);
#pragma unroll
                for (int ks = 0; ks < KC / 16; ++ks) {
                    const uint32_t o = ks * 256;
                    mma_f16(d, make_desc(aH + o, 128, 512), make_desc(bL + o, 128, 512), ks > 0 ? 1u : 0u);
                    mma_f16(d, make_desc(aL + o, 128, 512), make_desc(bH + o, 128, 512), 1u);
                }
#pragma unroll
                for (int ks = 0; ks < KC / 16; ++ks) {
                    const uint32_t o = ks * 256;
                    mma_f16(d, make_desc(aH + o, 128, 512), make_desc(bH + o, 128, 512), 1u);
                }
                mma_commit(smem_u32(&emptyA[s]));
                mma_commit(smem_u32(&accFull[a]));
                committed = ch + 1;
            }
        }
    } else {
        // ---------------------------------------------------------- workers
        float acc[64];
#pragma unroll
        for (int q = 0; q < 64; ++q) acc[q] = 0.f;
        const uint32_t trow = dtmem + ((uint32_t)(32 * warp) << 16);
        bool ok = true;
        for (int ch = 0; ch < nchunks && ok; ++ch) {
            const int a = ch % NACC;
            if (!ws_wait(smem_u32(&accFull[a]), (uint32_t)((ch / NACC) & 1), abort)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                uint32_t v[16];
                tmem_ld16(trow + (uint32_t)(a * TN + 16 * h), v);
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[16 * h + q] += __uint_as_float(v[q]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(smem_u32(&accEmpty[a]));
        }
        if (ok) {
            const int row = 32 * warp + lane;
            const int i = i0 + row;
            if (i < nrows) {
                const float ri = tcRinv[SYNTH ? rowBase[blockIdx.x] + row : tcOff[blockIdx.x] / (32 * nchunks) + row];
                if constexpr (SYNTH) {   // bvec[map][m][par][k], k = i
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        if (b0 + q < B) {
                            const float sc = ri * tinv[q];
                            alm[(((int64_t)(b0 + q) * (p + 1) + m) * 2 + par) * P2 + i] =
                                mk<float>(acc[q] * sc, acc[32 + q] * sc);
                        }
                } else if constexpr (DENSE) {   // beta[m][par][i][map]: the 32 maps side by side
                    cplx<float>* out = alm + (((int64_t)m * 2 + par) * P2 + i) * B + b0;
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        if (b0 + q < B) {
                            const float sc = ri * tinv[q];
                            out[q] = mk<float>(acc[q] * sc, acc[32 + q] * sc);
                        }
                } else {
                    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2 + m + c + 2 * (int64_t)i;
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        if (b0 + q < B) {
                            const float sc = ri * tinv[q];
                            alm[(int64_t)(b0 + q) * nalm + base] = mk<float>(acc[q] * sc, acc[32 + q] * sc);
                        }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (abort_) {
        if (tid == 0) {
            atomicExch(status, HPX_ERR_TIMEOUT);
            // copies issued but not seen by the MMA warp, and the last MMAs
            for (int q = seenA; q < issuedA; ++q)
                mbar_wait(smem_u32(&fullA[q % NSH]), (uint32_t)((q / NSH) & 1));
            if (committed > 0)
                mbar_wait(smem_u32(&accFull[(committed - 1) % NACC]), (uint32_t)(((committed - 1) / NACC) & 1));
        }
        __syncthreads();
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(dtmem), "r"(NACC * TN) : "memory");
}

// Plan time, FP32 tiles -> FP16 form in place (one block of 128 threads per
// tile, thread r = row r): the row's largest magnitude gives its scale s_r,
// 1 / s_r goes to rinv, and every chunk (all of it read before any of it is
// rewritten) becomes the hi block followed by the lo block of s_r M.
// rowsAll > 0: every tile belongs to a matrix of rowsAll rows (D, S^T), else to
// the chain (m, c) of the tile table.  tileNch / rowBase (both or neither):
// the tile's K-chunk count and the index of its first row scale, else
// ceil(P2 / 32) chunks and rows stored consecutively.
__global__ void __launch_bounds__(TM) tc_to_f16_kernel(float* __restrict__ Mt, const int64_t* __restrict__ tcOff,
                                                       const int* __restrict__ tiles, int P2, int L,
                                                       float* __restrict__ rinv, int rowsAll,
                                                       const int* __restrict__ tileNch,
                                                       const int64_t* __restrict__ rowBase) {
    const int m = tiles[3 * blockIdx.x], c = tiles[3 * blockIdx.x + 1], i0 = tiles[3 * blockIdx.x + 2];
    const int rp = (min(TM, (rowsAll > 0 ? rowsAll : chain_len(m, c, L)) - i0) + 7) & ~7;
    const int nchunks = tileNch ? tileNch[blockIdx.x] : (P2 + KC - 1) / KC;
    float* At = Mt + tcOff[blockIdx.x];
    const int r = threadIdx.x;
    const bool mine = r < rp;
    float mx = 0.f;
    if (mine)
        for (int ch = 0; ch < nchunks; ++ch) {
            const float* src = At + (int64_t)ch * rp * 32 + (r >> 3) * 256 + (r & 7) * 4;
            for (int kk = 0; kk < 8; ++kk) {
                const float4 v = *reinterpret_cast<const float4*>(src + kk * 32);
                mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
            }
        }
    const float sr = pow2_scale(mx, 14);
    if (mine) rinv[rowBase ? rowBase[blockIdx.x] + r : tcOff[blockIdx.x] / (32 * nchunks) + r] = 1.f / sr;
    for (int ch = 0; ch < nchunks; ++ch) {
        float* base = At + (int64_t)ch * rp * 32;
        float v[32];
        if (mine) {
            const float* src = base + (r >> 3) * 256 + (r & 7) * 4;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const float4 q = *reinterpret_cast<const float4*>(src + kk * 32);
                v[4 * kk] = q.x; v[4 * kk + 1] = q.y; v[4 * kk + 2] = q.z; v[4 * kk + 3] = q.w;
            }
        }
        __syncthreads();
        if (mine) {
            unsigned char* hb = reinterpret_cast<unsigned char*>(base) + (r >> 3) * 512 + (r & 7) * 16;
#pragma unroll
            for (int kc = 0; kc < 4; ++kc) {
                uint32_t h[4], l[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const HalfPair a = split_h(sr * v[8 * kc + 2 * e]), b = split_h(sr * v[8 * kc + 2 * e + 1]);
                    h[e] = pack_h(a.hi, b.hi);
                    l[e] = pack_h(a.lo, b.lo);
                }
                *reinterpret_cast<uint4*>(hb + kc * 128) = make_uint4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<uint4*>(hb + rp * 64 + kc * 128) = make_uint4(l[0], l[1], l[2], l[3]);
            }
        }
        __syncthreads();
    }
}

// Failure-path self-test: a wait on an mbarrier that nothing completes gives up
// after `spins` polls and reports like the operator kernel does.
__global__ void timeout_selftest_kernel(int* __restrict__ status, uint32_t spins) {
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x != 0) return;
    mbar_init(smem_u32(&mbar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(smem_u32(&mbar), 0u, spins)) atomicExch(status, HPX_ERR_TIMEOUT);
}

void launch_timeout_selftest(const hpx_plan_s* P, int spins, cudaStream_t s) {
    timeout_selftest_kernel<<<1, 32, 0, s>>>(P->d_status, (uint32_t)spins);
}

int prepare_fused_tc(hpx_plan_s* P) {
#if HPX_TC_F16
    const auto& g = P->g;
    const int64_t nch = (g.P2 + KC - 1) / KC;
    const int64_t rows = P->fused_bytes / 4 / (32 * nch);   // stored rows of all tiles
    const size_t rb = (size_t)rows * sizeof(float), bb = (size_t)g.B * (g.L + 1) * sizeof(float);
    const size_t pb = bpk_bytes(g.B, g.L, g.P2);
    if (cudaMalloc(&P->tcRinv, rb) != cudaSuccess || cudaMalloc(&P->bscale, bb) != cudaSuccess ||
        cudaMalloc(&P->bpk, pb) != cudaSuccess)
        return -1;
    cudaMemset(P->bpk, 0, pb);   // columns of maps past the batch stay zero
    P->bytes += (int64_t)(rb + bb + pb);
    P->fused_bytes += (int64_t)(rb + bb + pb);
    tc_to_f16_kernel<<<P->fused_ntiles, TM>>>((float*)P->fusedM, P->tcOff, P->fusedTiles, g.P2, g.L, P->tcRinv, 0,
                                              nullptr, nullptr);
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : -1;
#else
    (void)P;
    return 0;
#endif
}

void launch_fused_tc(const hpx_plan_s* P, float* alm, cudaStream_t s) {
    const auto& g = P->g;
    dim3 grid(P->fused_ntiles, (g.B + 31) / 32);
#if HPX_TC_F16
    const size_t smem_h = NSH * (TILE_A + TILE_BP);
    cudaFuncSetAttribute(fused_tc_ws_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_h);
    fused_tc_ws_kernel<0><<<grid, NTW, smem_h, s>>>((const unsigned char*)P->fusedM, P->tcOff, P->tcRinv,
                                                    P->fusedTiles, (const unsigned char*)P->bpk, P->bscale,
                                                    (cplx<float>*)alm, g.P2, g.p, g.L, g.B, g.nalm, P->d_status,
                                                    nullptr);
#else
    const size_t smem_t = NSA * TILE_A + 4 * TILE_B;
    cudaFuncSetAttribute(fused_tc_tmem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_t);
    fused_tc_tmem_kernel<<<grid, NT, smem_t, s>>>((const float*)P->fusedM, P->tcOff, P->fusedTiles,
                                                  (const cplx<float>*)P->bvec, (cplx<float>*)alm, g.P2, g.p, g.L,
                                                  g.B, g.nalm, P->d_status);
#endif
}

// D (FP32, [mpar][par][q][k], P2 x P2 per block) -> tile u of rows i0.. of
// block blk in the FP32 core-matrix layout of the operator tiles (K-chunks of
// rp x 32; rows and k past P2 zero).  One block of 128 threads per tile,
// thread = row.
__global__ void __launch_bounds__(TM) dense_tiles_kernel(const float* __restrict__ D, float* __restrict__ Mt,
                                                         const int64_t* __restrict__ tcOff,
                                                         const int* __restrict__ tiles, int P2) {
    const int blk = tiles[3 * blockIdx.x], i0 = tiles[3 * blockIdx.x + 2];
    const int rp = (min(TM, P2 - i0) + 7) & ~7;
    const int nchunks = (P2 + KC - 1) / KC;
    const int r = threadIdx.x;
    if (r >= rp) return;
    const int q = i0 + r;
    const float* src = D + ((size_t)blk * P2 + min(q, P2 - 1)) * P2;
    float* At = Mt + tcOff[blockIdx.x];
    for (int ch = 0; ch < nchunks; ++ch)
        for (int kk = 0; kk < KC; ++kk) {
            const int k = ch * KC + kk;
            const float v = (q < P2 && k < P2) ? src[k] : 0.f;
            At[(int64_t)ch * rp * 32 + (r >> 3) * 256 + (kk >> 2) * 32 + (r & 7) * 4 + (kk & 3)] = v;
        }
}

int prepare_dense_tc(hpx_plan_s* P) {
#if HPX_TC_F16
    const auto& g = P->g;
    const int nch = (g.P2 + KC - 1) / KC;
    const int nti = (g.P2 + TM - 1) / TM;
    // the 4 x nti distinct tiles of D, then one CTA tile per (m, par, row tile)
    std::vector<int> utiles;
    std::vector<int64_t> uoff;
    int64_t o = 0, rows = 0;
    for (int blk = 0; blk < 4; ++blk)
        for (int ti = 0; ti < nti; ++ti) {
            const int i0 = ti * TM, rp = (std::min(TM, g.P2 - i0) + 7) & ~7;
            utiles.insert(utiles.end(), {blk, 0, i0});
            uoff.push_back(o);
            o += (int64_t)nch * rp * 32;
            rows += rp;
        }
    std::vector<int> tiles;
    std::vector<int64_t> off;
    for (int m = 0; m <= g.L; ++m)
        for (int par = 0; par < 2; ++par)
            for (int ti = 0; ti < nti; ++ti) {
                tiles.insert(tiles.end(), {m, par, ti * TM});
                off.push_back(uoff[(size_t)((m & 1) * 2 + par) * nti + ti]);
            }
    int *du = nullptr, *dt = nullptr;
    int64_t *duo = nullptr, *dto = nullptr;
    const size_t bb = (size_t)g.B * (g.L + 1) * sizeof(float);
    bool ok = cudaMalloc(&P->dTC, (size_t)o * 4) == cudaSuccess &&
              cudaMalloc(&P->dRinv, (size_t)rows * 4) == cudaSuccess &&
              cudaMalloc(&du, utiles.size() * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&duo, uoff.size() * sizeof(int64_t)) == cudaSuccess &&
              cudaMalloc(&dt, tiles.size() * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&dto, off.size() * sizeof(int64_t)) == cudaSuccess &&
              (P->bscale || cudaMalloc(&P->bscale, bb) == cudaSuccess) &&
              (P->bpk || (cudaMalloc(&P->bpk, bpk_bytes(g.B, g.L, g.P2)) == cudaSuccess &&
                          cudaMemset(P->bpk, 0, bpk_bytes(g.B, g.L, g.P2)) == cudaSuccess));
    if (ok) {
        cudaMemcpy(du, utiles.data(), utiles.size() * sizeof(int), cudaMemcpyHostToDevice);
        cudaMemcpy(duo, uoff.data(), uoff.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
        cudaMemcpy(dt, tiles.data(), tiles.size() * sizeof(int), cudaMemcpyHostToDevice);
        cudaMemcpy(dto, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
        const int nu = (int)uoff.size();
        dense_tiles_kernel<<<nu, TM>>>((const float*)P->t.D, (float*)P->dTC, duo, du, g.P2);
        tc_to_f16_kernel<<<nu, TM>>>((float*)P->dTC, duo, du, g.P2, g.L, (float*)P->dRinv, g.P2, nullptr, nullptr);
        ok = cudaDeviceSynchronize() == cudaSuccess;
    }
    if (du) cudaFree(du);
    if (duo) cudaFree(duo);
    P->dTiles = dt;
    P->dTcOff = dto;
    P->dNtiles = (int)off.size();
    P->bytes += (int64_t)o * 4 + rows * 4 + (int64_t)bb + (int64_t)bpk_bytes(g.B, g.L, g.P2) +
                (int64_t)(tiles.size() * sizeof(int) + off.size() * 8);
    return ok ? 0 : -1;
#else
    (void)P;
    return 0;
#endif
}

void launch_dense_tc(const hpx_plan_s* P, cudaStream_t s) {
#if HPX_TC_F16
    const auto& g = P->g;
    dim3 grid(P->dNtiles, (g.B + 31) / 32);
    const size_t smem_h = NSH * (TILE_A + TILE_BP);
    cudaFuncSetAttribute(fused_tc_ws_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_h);
    fused_tc_ws_kernel<1><<<grid, NTW, smem_h, s>>>((const unsigned char*)P->dTC, P->dTcOff, (const float*)P->dRinv,
                                                    P->dTiles, (const unsigned char*)P->bpk, P->bscale,
                                                    (cplx<float>*)P->beta, g.P2, g.p, g.L, g.B, g.nalm, P->d_status,
                                                    nullptr);
#else
    (void)P;
    (void)s;
#endif
}

// S_{m,c} (row-major: chain row i, latitude mode k; n_alm x ldm) -> tiles of
// S^T: tile (m, c, k0) = rows k = k0.. (rp of them), K = the chain's rows in
// chunks of 32, in the FP32 core-matrix layout of the operator tiles (k past
// P2 and i past the chain zero).  One block of 128 threads per tile, thread =
// row; consecutive threads read consecutive k of one row of S.
__global__ void __launch_bounds__(TM) syn_tiles_kernel(const float* __restrict__ S, int ldm,
                                                       const int64_t* __restrict__ moff, float* __restrict__ Mt,
                                                       const int64_t* __restrict__ tcOff, const int* __restrict__ tiles,
                                                       int P2, int L) {
    const int m = tiles[3 * blockIdx.x], c = tiles[3 * blockIdx.x + 1], k0 = tiles[3 * blockIdx.x + 2];
    const int rp = (min(TM, P2 - k0) + 7) & ~7;
    const int nrows = chain_len(m, c, L);
    const int nch = (nrows + KC - 1) / KC;
    const int r = threadIdx.x;
    if (r >= rp) return;
    const int k = k0 + r;
    const float* A = S + moff[(size_t)m * 2 + c] * ldm;
    float* At = Mt + tcOff[blockIdx.x];
    for (int ch = 0; ch < nch; ++ch)
        for (int kk = 0; kk < KC; ++kk) {
            const int i = ch * KC + kk;
            const float v = (i < nrows && k < P2) ? A[(size_t)i * ldm + k] : 0.f;
            At[(int64_t)ch * rp * 32 + (r >> 3) * 256 + (kk >> 2) * 32 + (r & 7) * 4 + (kk & 3)] = v;
        }
}

// The synthesis' coefficients in the packed B layout: per (map b, order m) the
// two chains c (degrees m + c + 2i), each scaled by its own largest magnitude
// (recorded in scale[b][m][c]).  One block per (map, order), maps fastest.
__global__ void __launch_bounds__(256) pack_alm_kernel(const cplx<float>* __restrict__ alm,
                                                       unsigned char* __restrict__ bpk, float* __restrict__ scale,
                                                       int L, int P2, int64_t nalm) {
    __shared__ float2 red32[32];
    const int b = blockIdx.x, m = blockIdx.y;
    const int nch = (P2 + KC - 1) / KC;
    const cplx<float>* a = alm + (int64_t)b * nalm + (int64_t)m * (2 * L + 1 - m) / 2 + m;   // a[l - m]
    const int n0 = chain_len(m, 0, L), n1 = chain_len(m, 1, L);
    float mx0 = 0.f, mx1 = 0.f;
    for (int j = threadIdx.x; j <= L - m; j += blockDim.x) {
        const cplx<float> v = a[j];
        const float x = fmaxf(fabsf(v.r), fabsf(v.i));
        if (j & 1) mx1 = fmaxf(mx1, x);
        else mx0 = fmaxf(mx0, x);
    }
    const float2 mx = block_max2(make_float2(mx0, mx1), red32);
    if (threadIdx.x < 2) scale[((int64_t)b * (L + 1) + m) * 2 + threadIdx.x] = threadIdx.x ? mx.y : mx.x;
    pack_half(bpk, b, m, 0, L, nch, pow2_scale(mx.x, 13),
              [&](int i) { return i < n0 ? a[2 * i] : mk<float>(0.f, 0.f); }, threadIdx.x, blockDim.x);
    pack_half(bpk, b, m, 1, L, nch, pow2_scale(mx.y, 13),
              [&](int i) { return i < n1 ? a[2 * i + 1] : mk<float>(0.f, 0.f); }, threadIdx.x, blockDim.x);
}

int prepare_synth_tc(hpx_plan_s* P) {
#if HPX_TC_F16
    const auto& g = P->g;
    std::vector<int> tiles, nchs;
    std::vector<int64_t> off, rbase;
    int64_t o = 0, rows = 0;
    for (int m = 0; m <= g.L; ++m)
        for (int c = 0; c < 2; ++c) {
            const int nch = (chain_len(m, c, g.L) + KC - 1) / KC;
            for (int k0 = 0; k0 < g.P2; k0 += TM) {
                const int rp = (std::min(TM, g.P2 - k0) + 7) & ~7;
                tiles.insert(tiles.end(), {m, c, k0});
                nchs.push_back(nch);
                off.push_back(o);
                rbase.push_back(rows);
                o += (int64_t)nch * rp * 32;
                rows += rp;
            }
        }
    const size_t sb = (size_t)g.B * (g.L + 1) * 2 * sizeof(float), pb = bpk_bytes(g.B, g.L, g.P2);
    int *dt = nullptr, *dn = nullptr;
    int64_t *doff = nullptr, *drb = nullptr;
    bool ok = cudaMalloc(&P->synT, (size_t)std::max<int64_t>(o, 1) * 4) == cudaSuccess &&
              cudaMalloc(&P->synRinv, (size_t)rows * 4) == cudaSuccess &&
              cudaMalloc(&dt, tiles.size() * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&dn, nchs.size() * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&doff, off.size() * sizeof(int64_t)) == cudaSuccess &&
              cudaMalloc(&drb, rbase.size() * sizeof(int64_t)) == cudaSuccess &&
              cudaMalloc(&P->synScale, sb) == cudaSuccess && cudaMalloc(&P->synBpk, pb) == cudaSuccess;
    P->synTiles = dt;
    P->synNch = dn;
    P->synOff = doff;
    P->synRowBase = drb;
    if (!ok) return -1;
    cudaMemcpy(dt, tiles.data(), tiles.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(dn, nchs.data(), nchs.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(doff, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    cudaMemcpy(drb, rbase.data(), rbase.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    cudaMemset(P->synBpk, 0, pb);   // columns of maps past the batch stay zero
    P->synNtiles = (int)off.size();
    const int nt = P->synNtiles;
    syn_tiles_kernel<<<nt, TM>>>((const float*)P->synM, P->fused_ldm, P->fusedOff, (float*)P->synT, doff, dt,
                                 g.P2, g.L);
    tc_to_f16_kernel<<<nt, TM>>>((float*)P->synT, doff, dt, g.P2, g.L, (float*)P->synRinv, g.P2, dn, drb);
    P->bytes += o * 4 + rows * 4 + (int64_t)(sb + pb) + (int64_t)(tiles.size() + nchs.size()) * 4 +
                (int64_t)(off.size() + rbase.size()) * 8;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : -1;
#else
    (void)P;
    return 0;
#endif
}

void launch_synth_tc(const hpx_plan_s* P, const float* alm, cudaStream_t s) {
#if HPX_TC_F16
    const auto& g = P->g;
    pack_alm_kernel<<<dim3(g.B, g.L + 1), 256, 0, s>>>((const cplx<float>*)alm, (unsigned char*)P->synBpk,
                                                       (float*)P->synScale, g.L, g.P2, g.nalm);
    dim3 grid(P->synNtiles, (g.B + 31) / 32);
    const size_t smem_h = NSH * (TILE_A + TILE_BP);
    cudaFuncSetAttribute(fused_tc_ws_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_h);
    fused_tc_ws_kernel<2><<<grid, NTW, smem_h, s>>>((const unsigned char*)P->synT, P->synOff,
                                                    (const float*)P->synRinv, P->synTiles,
                                                    (const unsigned char*)P->synBpk, (const float*)P->synScale,
                                                    (cplx<float>*)P->bvec, g.P2, g.p, g.L, g.B, g.nalm, P->d_status,
                                                    P->synRowBase);
#else
    (void)P;
    (void)alm;
    (void)s;
#endif
}

}  // namespace hpx
