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
    for (int s = 1; s <= logn; ++s) {
        const int half = 1 << (s - 1);
        const int tstride = twlen >> s;   // e^{-2 pi i pos / 2^s} = tw[pos * twlen / 2^s]
        for (int k = tid; k < (n >> 1); k += nt) {
            const int pos = k & (half - 1);
            const int i0 = ((k >> (s - 1)) << s) + pos;
            const int i1 = i0 + half;
            cplx<T> w = tw[pos * tstride];
            if (inverse) w.i = -w.i;
            const cplx<T> u = a[i0];
            const cplx<T> v = mul(a[i1], w);
            a[i0] = add(u, v);
            a[i1] = sub(u, v);
        }
        __syncthreads();
    }
}

}  // namespace hpx
