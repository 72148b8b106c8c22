// Per-order operators on the 5th-generation tensor cores (tcgen05, TMEM).
//
// The contraction a_{m+c+2i}^m[map] = sum_k M_{m,c}[i][k] b[map][m][par][k] of
// k_fused.cu, for FP32 plans, as 3xTF32 MMAs: every operand x is split into
// x_hi = x with the low 13 mantissa bits cleared (exactly a TF32 number) and
// x_lo = x - x_hi, and the product is accumulated as
//     A_hi B_hi + A_hi B_lo + A_lo B_hi
// in FP32 in tensor memory (the dropped A_lo B_lo term is below 2^-22 of the
// product).  One CTA (4 warps) computes a tile of 128 rows (degrees of one
// chain) x 64 real columns (re, im of 32 maps) over K = P2 in chunks of 32:
//   * all threads load the FP32 chunk of M (16 KB) and of b (8 KB), split it and
//     store hi / lo copies in shared memory in the K-major, no-swizzle core-matrix
//     layout of the MMA (8 rows x 16 bytes per core matrix; core matrices
//     adjacent in K are 128 bytes apart, 8-row groups 1 KB apart);
//   * one thread issues 4 K-steps x 3 tcgen05.mma (M=128, N=64, K=8) and commits
//     them to an mbarrier; the CTA waits on it before the next chunk overwrites
//     the tiles (several CTAs per SM keep the loads and the MMAs overlapped);
//   * the epilogue reads the 128 x 64 FP32 accumulator from TMEM with
//     tcgen05.ld (warp w owns TMEM lanes 32w..32w+31) and writes the coefficients.
// Every wait is bounded: on timeout the CTA records HPX_ERR_TIMEOUT in the
// plan's status word and returns after releasing its tensor memory.
#include <cstdint>

#include "plan.h"
#include "plan_math.h"

namespace hpx {

namespace {

constexpr int TM = 128;          // rows per tile (MMA M)
constexpr int TN = 64;           // real columns per tile (MMA N): 32 maps x (re, im)
constexpr int KC = 32;           // K per chunk
constexpr int TILE_A = TM * KC * 4;   // bytes of one A copy (16 KB)
constexpr int TILE_B = TN * KC * 4;   // bytes of one B copy (8 KB)
constexpr uint32_t kSpinLimit = 1u << 26;

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

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(dtmem), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// Bounded wait for the given phase parity; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
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
    }
    return false;
}

__device__ __forceinline__ uint32_t split_hi(float x) { return __float_as_uint(x) & 0xFFFFE000u; }

// byte offset of (row r, k) in a K-major no-swizzle tile with KC = 32
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

}  // namespace

__global__ void __launch_bounds__(128) fused_tc_kernel(const float* __restrict__ M, const int64_t* __restrict__ moff,
                                                       const int* __restrict__ tiles,
                                                       const cplx<float>* __restrict__ bvec,
                                                       cplx<float>* __restrict__ alm, int P2, int ldm, int p, int L,
                                                       int B, int64_t nalm, int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* Ahi = smem;
    unsigned char* Alo = smem + TILE_A;
    unsigned char* Bhi = smem + 2 * TILE_A;
    unsigned char* Blo = smem + 2 * TILE_A + TILE_B;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = tiles[3 * blockIdx.x], c = tiles[3 * blockIdx.x + 1], i0 = tiles[3 * blockIdx.x + 2];
    const int par = ((m & 1) + c) & 1;
    const int nrows = chain_len(m, c, L);
    const int b0 = blockIdx.y * (TN / 2);
    const float* A = M + moff[(size_t)m * 2 + c] * ldm;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&mbar), 1);
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t dtmem = tmem_base;

    const int nchunks = (P2 + KC - 1) / KC;
    uint32_t phase = 0;
    for (int ch = 0; ch < nchunks; ++ch) {
        const int k0 = ch * KC;
        // A chunk: 128 rows x 8 float4 (coalesced along k)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int idx = tid + 128 * j;
            const int r = idx >> 3, kq = idx & 7;
            const int i = i0 + r;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < nrows && k0 + 4 * kq < ldm) v = *reinterpret_cast<const float4*>(A + (size_t)i * ldm + k0 + 4 * kq);
            uint4 hi = make_uint4(split_hi(v.x), split_hi(v.y), split_hi(v.z), split_hi(v.w));
            float4 lo = make_float4(v.x - __uint_as_float(hi.x), v.y - __uint_as_float(hi.y),
                                    v.z - __uint_as_float(hi.z), v.w - __uint_as_float(hi.w));
            const uint32_t off = tile_off(r, 4 * kq);
            *reinterpret_cast<uint4*>(Ahi + off) = hi;
            *reinterpret_cast<float4*>(Alo + off) = lo;
        }
        // B chunk: 32 maps x 32 complex (16 float4 per map); re -> row 2b, im -> row 2b+1
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int idx = tid + 128 * j;
            const int bl = idx >> 4, kq = idx & 15;   // complex k = k0 + 2 kq, k0 + 2 kq + 1
            const int b = b0 + bl, k = k0 + 2 * kq;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (b < B && k < P2) {
                const float* src = reinterpret_cast<const float*>(bvec + (((int64_t)b * (p + 1) + m) * 2 + par) * P2 + k);
                v.x = src[0];
                v.y = src[1];
                if (k + 1 < P2) { v.z = src[2]; v.w = src[3]; }
            }
            const uint32_t offr = tile_off(2 * bl, 2 * kq), offi = tile_off(2 * bl + 1, 2 * kq);
            const uint32_t hr0 = split_hi(v.x), hr1 = split_hi(v.z), hi0 = split_hi(v.y), hi1 = split_hi(v.w);
            *reinterpret_cast<uint2*>(Bhi + offr) = make_uint2(hr0, hr1);
            *reinterpret_cast<uint2*>(Bhi + offi) = make_uint2(hi0, hi1);
            *reinterpret_cast<float2*>(Blo + offr) = make_float2(v.x - __uint_as_float(hr0), v.z - __uint_as_float(hr1));
            *reinterpret_cast<float2*>(Blo + offi) = make_float2(v.y - __uint_as_float(hi0), v.w - __uint_as_float(hi1));
        }
        // generic-proxy smem writes -> visible to the tensor core
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t aH = smem_u32(Ahi), aL = smem_u32(Alo), bH = smem_u32(Bhi), bL = smem_u32(Blo);
#pragma unroll
            for (int ks = 0; ks < KC / 8; ++ks) {
                const uint32_t o = ks * 256;   // 8 k = two core matrices along K
                const uint64_t dAh = make_desc(aH + o, 128, 1024), dAl = make_desc(aL + o, 128, 1024);
                const uint64_t dBh = make_desc(bH + o, 128, 1024), dBl = make_desc(bL + o, 128, 1024);
                mma_tf32(dtmem, dAh, dBh, (ch > 0 || ks > 0) ? 1u : 0u);
                mma_tf32(dtmem, dAh, dBl, 1u);
                mma_tf32(dtmem, dAl, dBh, 1u);
            }
            mma_commit(smem_u32(&mbar));
        }
        // the tiles are reused by the next chunk: wait for these MMAs
        if (!mbar_wait(smem_u32(&mbar), phase)) {
            if (lane == 0) atomicExch(&failed, 1);
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (failed) break;
    }

    if (!failed) {
        // epilogue: row 32 warp + lane of the tile, 64 FP32 columns
        uint32_t v[64];
        const uint32_t taddr = dtmem + ((uint32_t)(32 * warp) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
            "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
            "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]),
              "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]),
              "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]),
              "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]),
              "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int i = i0 + 32 * warp + lane;
        if (i < nrows) {
            const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2 + m + c + 2 * (int64_t)i;
#pragma unroll
            for (int bl = 0; bl < TN / 2; ++bl) {
                const int b = b0 + bl;
                if (b < B) alm[(int64_t)b * nalm + base] = mk<float>(__uint_as_float(v[2 * bl]), __uint_as_float(v[2 * bl + 1]));
            }
        }
    } else if (tid == 0) {
        atomicExch(status, HPX_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(dtmem), "r"(TN) : "memory");
}

void launch_fused_tc(const hpx_plan_s* P, float* alm, cudaStream_t s) {
    const auto& g = P->g;
    const size_t smem = 2 * TILE_A + 2 * TILE_B;
    cudaFuncSetAttribute(fused_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid(P->fused_ntiles, (g.B + 31) / 32);
    fused_tc_kernel<<<grid, 128, smem, s>>>((const float*)P->fusedM, P->fusedOff, P->fusedTiles,
                                            (const cplx<float>*)P->bvec, (cplx<float>*)alm, g.P2, P->fused_ldm, g.p,
                                            g.L, g.B, g.nalm, P->d_status);
}

}  // namespace hpx
