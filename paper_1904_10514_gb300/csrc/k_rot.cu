// Fourier-to-spherical-harmonic conversion, part 1 (Sec. 3.3): the connection
// between normalised associated Legendre functions of orders m' and m'+2 is a
// product of Givens rotations, so the order-m coefficients follow from the
// order-0 (m even) or order-1 (m odd) coefficients by m/2 rotation sweeps.
//
// In the analysis direction one sweep maps the chain of order-m' coefficients
// v_0..v_n (degrees m'+c+2i, c = parity chain) to the order-(m'+2) chain
// w_0..w_{n-1}:
//     carry = v_0;  for i = 1..n: (w_{i-1}, carry) = (c_i carry + s_i v_i,
//                                                     -s_i carry + c_i v_i)
// and the last carry is dropped (it is the component outside the order-(m'+2)
// span).  The angles are FP64-built at plan time from the QR factorisation of
// the tridiagonal multiplication-by-sin^2 operator.
//
// Kernel layout: one block per (m, group of G maps), one warp per parity chain.
// Lane s of a warp applies stage s0 + s of the current pass of 32 stages; the
// chain streams through the lanes as a wavefront (lane s runs two steps behind
// lane s - 1) and each rotated value is handed to the next stage with a warp
// shuffle.  Lane 0 reads the chain from shared memory and the last lane writes
// the pass's output chain back in place.  Each lane carries 2G real values
// (re, im of G maps) that share one angle load.
#include "plan.h"
#include "plan_math.h"

namespace hpx {

template <class T, int G>
__global__ void __launch_bounds__(64) rot_kernel(const cplx<T>* __restrict__ beta, cplx<T>* __restrict__ alm,
                                                 const int64_t* __restrict__ angOff,
                                                 const cplx<T>* __restrict__ ang, int p, int P2, int L, int B,
                                                 int64_t nalm, int nmax) {
    constexpr int V = 2 * G;
    extern __shared__ unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = warp;   // parity chain
    T* buf = reinterpret_cast<T*>(smem_raw) + (size_t)warp * nmax * V;
    const int m = blockIdx.x;
    const int b0 = blockIdx.y * G;
    const int m0 = m & 1;
    const int S = (m - m0) >> 1;
    const int N0 = chain_len(m0, c, L);

    for (int idx = lane; idx < N0; idx += 32) {
        const int l = m0 + c + 2 * idx;
        const int par = l & 1, q = l >> 1;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            cplx<T> v = mk<T>(T(0), T(0));
            if (b0 + g < B) v = beta[(((int64_t)(b0 + g) * (p + 1) + m) * 2 + par) * P2 + q];
            buf[idx * V + 2 * g] = v.r;
            buf[idx * V + 2 * g + 1] = v.i;
        }
    }
    __syncwarp();

    int ncur = N0;
    for (int s0 = 0; s0 < S && ncur > 0; s0 += 32) {
        const int nst = min(32, S - s0);
        const int last = nst - 1;
        const int nrot = ncur - 1 - lane;   // rotations of this lane's stage
        const bool active = lane < nst;
        const cplx<T>* an = ang + (active ? angOff[(size_t)(m0 + 2 * (s0 + lane)) * 2 + c] : 0);
        T carry[V], in[V], out[V];
#pragma unroll
        for (int v = 0; v < V; ++v) { carry[v] = T(0); in[v] = T(0); out[v] = T(0); }
        const int tend = ncur + last;
        for (int t = 0; t < tend; ++t) {
            const int i = t - 2 * lane;
            if (lane == 0 && i >= 0 && i < ncur) {
#pragma unroll
                for (int v = 0; v < V; ++v) in[v] = buf[i * V + v];
            }
            if (active && i >= 0 && i <= nrot) {
                if (i == 0) {
#pragma unroll
                    for (int v = 0; v < V; ++v) carry[v] = in[v];
                } else {
                    const cplx<T> cs = an[i - 1];
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const T o = cs.r * carry[v] + cs.i * in[v];
                        carry[v] = cs.r * in[v] - cs.i * carry[v];
                        out[v] = o;
                    }
                    if (lane == last) {
#pragma unroll
                        for (int v = 0; v < V; ++v) buf[(i - 1) * V + v] = out[v];
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) in[v] = __shfl_up_sync(0xffffffffu, out[v], 1);
            __syncwarp();
        }
        ncur -= nst;
    }
    __syncwarp();

    for (int idx = lane; idx < ncur; idx += 32) {
        const int l = m + c + 2 * idx;
        const int64_t o = (int64_t)m * (2 * L + 1 - m) / 2 + l;
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (b0 + g < B) alm[(int64_t)(b0 + g) * nalm + o] = mk<T>(buf[idx * V + 2 * g], buf[idx * V + 2 * g + 1]);
    }
}

template <class T>
void launch_rot(const hpx_plan_s* P, T* alm, cudaStream_t s) {
    const auto& g = P->g;
    const int nmax = g.L / 2 + 1;
    if (g.B >= 4) {
        constexpr int G = 4;
        const size_t smem = (size_t)2 * nmax * 2 * G * sizeof(T);
        cudaFuncSetAttribute(rot_kernel<T, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dim3 grid(g.L + 1, (g.B + G - 1) / G);
        rot_kernel<T, G><<<grid, 64, smem, s>>>((const cplx<T>*)P->beta, (cplx<T>*)alm, P->t.angOff,
                                                (const cplx<T>*)P->t.ang, g.p, g.P2, g.L, g.B, g.nalm, nmax);
    } else {
        constexpr int G = 1;
        const size_t smem = (size_t)2 * nmax * 2 * G * sizeof(T);
        cudaFuncSetAttribute(rot_kernel<T, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dim3 grid(g.L + 1, g.B);
        rot_kernel<T, G><<<grid, 64, smem, s>>>((const cplx<T>*)P->beta, (cplx<T>*)alm, P->t.angOff,
                                                (const cplx<T>*)P->t.ang, g.p, g.P2, g.L, g.B, g.nalm, nmax);
    }
}

template void launch_rot<float>(const hpx_plan_s*, float*, cudaStream_t);
template void launch_rot<double>(const hpx_plan_s*, double*, cudaStream_t);

}  // namespace hpx
