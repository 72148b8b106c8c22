// FP16 pairs of FP32 numbers for the tensor-core contractions, and the packed
// layout of the right-hand sides b that those kernels read by bulk copy.
//
// After a power-of-two scaling x' = s x, hi = fp16(x') and lo = fp16(x' - hi)
// (x' - hi is exact in FP32) carry x' to |x' - hi - lo| <= 2^-22 |x'| while both
// are FP16 normal numbers; the products hi*lo + lo*hi + hi*hi of two such pairs
// are exact in an FP32 accumulator.
//
// Packed b: for map tile mt (32 maps), order m, parity par of the latitude
// index j and K-chunk ch (32 consecutive k = j >> 1) one block of kBpkChunk
// bytes: the hi copy, then the lo copy, each 64 columns x 32 k in the K-major,
// no-swizzle core-matrix order of tcgen05 (core matrix = 8 columns x 8 halves
// of 16 bytes each; 8-column groups 512 bytes apart, core matrices adjacent in
// K 128 bytes apart); columns 0-31 are the real parts of the tile's maps,
// columns 32-63 their imaginary parts.  Columns of maps past the batch stay
// zero (the buffer is cleared at plan time); k past the column is written as
// zero.  Blocks are ordered [mt][m][par][ch].
#pragma once
#include <cuda_fp16.h>

#include <cstdint>

#include "common.cuh"

namespace hpx {

struct HalfPair {
    __half hi, lo;
};
__device__ __forceinline__ HalfPair split_h(float x) {
    const __half h = __float2half_rn(x);
    return HalfPair{h, __float2half_rn(x - __half2float(h))};
}
// two halves in one 32-bit word, the first one at the lower address
__device__ __forceinline__ uint32_t pack_h(__half a, __half b) {
    return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

constexpr int kBpkChunk = 8192;   // bytes of one packed b chunk (hi + lo)

inline size_t bpk_bytes(int B, int L, int P2) {
    return (size_t)((B + 31) / 32) * (size_t)(L + 1) * 2 * (size_t)((P2 + 31) / 32) * kBpkChunk;
}

// One step of the packing: 8 consecutive k = 8 g8 .. 8 g8 + 7 of one half
// (parity or chain) of a column, val(k) the complex value (zero past the half's
// length), scaled by sc before the split; four 16-byte stores (hi and lo of the
// real and of the imaginary parts) into the half's blocks at `half`, column
// offset offr.
template <class V>
__device__ __forceinline__ void pack_group(unsigned char* __restrict__ half, int offr, int g8, float sc, V val) {
    uint32_t hr[4], lr[4], hm[4], lm[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int k = 8 * g8 + 2 * e;
        const cplx<float> v0 = val(k), v1 = val(k + 1);
        // the pairs of two consecutive k at once (the same roundings as split_h)
        const float2 xr = make_float2(sc * v0.r, sc * v1.r), xi = make_float2(sc * v0.i, sc * v1.i);
        const __half2 hR = __float22half2_rn(xr), hI = __float22half2_rn(xi);
        const float2 fR = __half22float2(hR), fI = __half22float2(hI);
        const __half2 lR = __float22half2_rn(make_float2(xr.x - fR.x, xr.y - fR.y));
        const __half2 lI = __float22half2_rn(make_float2(xi.x - fI.x, xi.y - fI.y));
        hr[e] = *reinterpret_cast<const uint32_t*>(&hR);
        lr[e] = *reinterpret_cast<const uint32_t*>(&lR);
        hm[e] = *reinterpret_cast<const uint32_t*>(&hI);
        lm[e] = *reinterpret_cast<const uint32_t*>(&lI);
    }
    unsigned char* blk = half + (int64_t)(g8 >> 2) * kBpkChunk + (g8 & 3) * 128 + offr;
    *reinterpret_cast<uint4*>(blk) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
    *reinterpret_cast<uint4*>(blk + 4096) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
    *reinterpret_cast<uint4*>(blk + 2048) = make_uint4(hm[0], hm[1], hm[2], hm[3]);
    *reinterpret_cast<uint4*>(blk + 4096 + 2048) = make_uint4(lm[0], lm[1], lm[2], lm[3]);
}

// First byte of half h (0 or 1) of column (map b, order m); nch K-chunks per half.
__device__ __forceinline__ unsigned char* packed_half(unsigned char* bpk, int b, int m, int h, int L, int nch) {
    return bpk + ((((int64_t)(b >> 5) * (L + 1) + m) * 2 + h) * nch) * kBpkChunk;
}
__device__ __forceinline__ int packed_col_offset(int b) { return ((b & 31) >> 3) * 512 + (b & 7) * 16; }

// Half h of column (map b, order m) by the nt threads tid, with its own scale.
template <class V>
__device__ __forceinline__ void pack_half(unsigned char* __restrict__ bpk, int b, int m, int h, int L, int nch,
                                          float sc, V val, int tid, int nt) {
    unsigned char* half = packed_half(bpk, b, m, h, L, nch);
    const int offr = packed_col_offset(b);
    for (int g8 = tid; g8 < nch * 4; g8 += nt) pack_group(half, offr, g8, sc, val);
}

// Both parities of column (map b, order m) with one scale: val(par, k).
template <class V>
__device__ __forceinline__ void pack_column(unsigned char* __restrict__ bpk, int b, int m, int L, int P2, float sc,
                                            V val, int tid, int nt) {
    const int nch = (P2 + 31) >> 5;
    const int offr = packed_col_offset(b);
    for (int gi = tid; gi < 8 * nch; gi += nt) {
        const int par = gi / (4 * nch), g8 = gi - par * (4 * nch);
        pack_group(packed_half(bpk, b, m, par, L, nch), offr, g8, sc, [&](int k) { return val(par, k); });
    }
}

// Largest of (v.x, v.y) over the block, each component on its own (every
// thread passes its partials; blockDim a multiple of 32, at most 1024).  Ends
// with a barrier.
__device__ __forceinline__ float2 block_max2(float2 v, float2* red32) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x = fmaxf(v.x, __shfl_xor_sync(0xffffffffu, v.x, o));
        v.y = fmaxf(v.y, __shfl_xor_sync(0xffffffffu, v.y, o));
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) red32[w] = v;
    __syncthreads();
    float2 r = make_float2(0.f, 0.f);
    for (int q = 0; q < nw; ++q) r = make_float2(fmaxf(r.x, red32[q].x), fmaxf(r.y, red32[q].y));
    __syncthreads();
    return r;
}

// Largest of v over the block (every thread passes its partial; blockDim a
// multiple of 32, at most 1024).  Ends with a barrier.
__device__ __forceinline__ float block_max(float v, float* red32) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red32[w] = v;
    __syncthreads();
    float r = 0.f;
    for (int q = 0; q < nw; ++q) r = fmaxf(r, red32[q]);
    __syncthreads();
    return r;
}

}  // namespace hpx
