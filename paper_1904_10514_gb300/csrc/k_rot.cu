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
// Kernel layout.  One warp per (m, parity chain c, group of 32 real columns),
// one lane per real column (re or im of one map).  A pass applies K consecutive
// sweeps at once as a wavefront held in registers: at time step t, stage k
// performs its rotation i = t - 2k, reading the value stage k-1 produced at the
// previous step, so the K rotations of a step are independent (ILP = K) and
// no data crosses lanes.  Stage 0 reads the chain from global memory (one
// coalesced 128-byte row per step); the last stage writes its output back in
// place (output index < input index, same lane).  The K angles of a step are
// the same for all lanes and come from a pre-skewed table (idle slots hold the
// rotation (1, 0), which only moves the input into the carry), so the inner
// loop has no branches.  m/2 sweeps take passes of 32 stages and then
// 16, 8, 4, 2, 1.
#include "plan.h"
#include "plan_math.h"
#include "sweep.cuh"

namespace hpx {

// Ring slots per warp of the staged form (sweep_pass_staged): copies run RB - 1
// steps ahead of their use.
constexpr int kRotRing = 8;

// FP32: the same work with the angle rows and chain inputs staged through
// shared memory ahead of use (sweep_pass_staged); every lane of a warp runs
// the passes (lanes without a map neither load nor store chain values).
template <int KMAX>
__global__ void __launch_bounds__(64, (KMAX == 32 ? 6 : 10)) rot_staged_kernel(cplx<float>* __restrict__ beta2, cplx<float>* __restrict__ alm,
                                                        const int64_t* __restrict__ skOff,
                                                        const cplx<float>* __restrict__ skew, int nq, int P2, int L,
                                                        int B, int64_t nalm, int ngroups, int nitems) {
    constexpr int SL = SweepRing<kRotRing>::kSlot;
    __shared__ __align__(16) cplx<float> rings[2][kRotRing * SL];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nitems) return;   // whole warps leave together (nitems counts warps)
    cplx<float>* ring = rings[(threadIdx.x >> 5) & 1];
    const int g = warp % ngroups;
    const int c = (warp / ngroups) & 1;
    const int m = L - warp / (2 * ngroups);
    const int m0 = m & 1;
    const int S = (m - m0) >> 1;
    const int col = 32 * g + lane;
    const bool live = col < B;
    const int par = (m0 + c) & 1;
    const int q0 = (m0 == 1 && c == 1) ? 1 : 0;
    cplx<float>* chain = beta2 + (((int64_t)m * 2 + par) * P2 + q0) * B + (live ? col : 0);
    const int64_t ldc = B;
    int n = chain_len(m0, c, L);
    int s0 = 0;
    auto block = [&](int s) {
        return skew + (skOff[(size_t)(m0 * 2 + c) * nq + (s >> 5)] + 2 * (s & 31)) * 32;
    };
    while (S - s0 >= KMAX && n > 0) {
        sweep_pass_staged<float, KMAX, kRotRing>(chain, ldc, n, live, block(s0), s0 & 31, ring);
        n -= KMAX;
        s0 += KMAX;
    }
#define HPX_SUBPASS(KK)                                                                   \
    if (KK < KMAX && S - s0 >= KK && n > 0) {                                             \
        sweep_pass_staged<float, KK, kRotRing>(chain, ldc, n, live, block(s0), s0 & 31, ring); \
        n -= KK;                                                                          \
        s0 += KK;                                                                         \
    }
    HPX_SUBPASS(16)
    HPX_SUBPASS(8)
    HPX_SUBPASS(4)
    HPX_SUBPASS(2)
    HPX_SUBPASS(1)
#undef HPX_SUBPASS
    if (!live) return;
    cplx<float>* out = alm + (int64_t)col * nalm;
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2 + m + c;
    for (int i = 0; i < n; ++i) out[base + 2 * i] = chain[(int64_t)i * ldc];
}

// FP32, one real column per lane (sweep_pass_staged_real): warp = (m, chain c,
// group of 32 real columns: re and im of 16 maps), so a batch of B maps fills
// 2B lanes.  Output: the lane's part of a_{m+c+2i}^m.
template <int KMAX>
__global__ void __launch_bounds__(64, 8) rot_staged_real_kernel(cplx<float>* __restrict__ beta2,
                                                               cplx<float>* __restrict__ alm,
                                                               const int64_t* __restrict__ skOff,
                                                               const cplx<float>* __restrict__ skew, int nq, int P2,
                                                               int L, int B, int64_t nalm, int ngroups, int nitems) {
    constexpr int SL = SweepRing<kRotRing>::kSlot;
    __shared__ __align__(16) cplx<float> rings[2][kRotRing * SL];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nitems) return;   // whole warps leave together (nitems counts warps)
    cplx<float>* ring = rings[(threadIdx.x >> 5) & 1];
    const int g = warp % ngroups;
    const int c = (warp / ngroups) & 1;
    const int m = L - warp / (2 * ngroups);
    const int m0 = m & 1;
    const int S = (m - m0) >> 1;
    const int rc = 32 * g + lane;   // real column: 2 map + part
    const bool live = rc < 2 * B;
    const int par = (m0 + c) & 1;
    const int q0 = (m0 == 1 && c == 1) ? 1 : 0;
    float* chain = reinterpret_cast<float*>(beta2 + (((int64_t)m * 2 + par) * P2 + q0) * B) + (live ? rc : 0);
    const int64_t ldc = 2 * (int64_t)B;
    int n = chain_len(m0, c, L);
    int s0 = 0;
    auto block = [&](int s) {
        return skew + (skOff[(size_t)(m0 * 2 + c) * nq + (s >> 5)] + 2 * (s & 31)) * 32;
    };
    while (S - s0 >= KMAX && n > 0) {
        sweep_pass_staged_real<KMAX, kRotRing>(chain, ldc, n, live, block(s0), s0 & 31, ring);
        n -= KMAX;
        s0 += KMAX;
    }
#define HPX_SUBPASS(KK)                                                                      \
    if (KK < KMAX && S - s0 >= KK && n > 0) {                                                \
        sweep_pass_staged_real<KK, kRotRing>(chain, ldc, n, live, block(s0), s0 & 31, ring); \
        n -= KK;                                                                             \
        s0 += KK;                                                                            \
    }
    HPX_SUBPASS(16)
    HPX_SUBPASS(8)
    HPX_SUBPASS(4)
    HPX_SUBPASS(2)
    HPX_SUBPASS(1)
#undef HPX_SUBPASS
    if (!live) return;
    float* out = reinterpret_cast<float*>(alm + (int64_t)(rc >> 1) * nalm) + (rc & 1);
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2 + m + c;
    for (int i = 0; i < n; ++i) out[2 * (base + 2 * i)] = chain[(int64_t)i * ldc];
}

template <class T, int KMAX>
__global__ void __launch_bounds__(64) rot_kernel(cplx<T>* __restrict__ beta2, cplx<T>* __restrict__ alm,
                                                  const int64_t* __restrict__ skOff,
                                                  const cplx<T>* __restrict__ skew, int nq, int P2, int L,
                                                  int B, int64_t nalm, int ngroups, int nitems) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nitems) return;
    // heaviest orders first: item -> (m descending, chain, column group)
    const int g = warp % ngroups;
    const int c = (warp / ngroups) & 1;
    const int m = L - warp / (2 * ngroups);
    const int m0 = m & 1;
    const int S = (m - m0) >> 1;
    const int ncol = B;                 // one complex column per map
    const int col = 32 * g + lane;      // map index
    const bool live = col < ncol;
    // chain c of order m0 sits in parity block par at rows q0, q0+1, ...
    const int par = (m0 + c) & 1;
    const int q0 = (m0 == 1 && c == 1) ? 1 : 0;
    cplx<T>* chain = beta2 + (((int64_t)m * 2 + par) * P2 + q0) * ncol + (live ? col : 0);
    const int64_t ldc = ncol;
    int n = chain_len(m0, c, L);
    int s0 = 0;
    // A pass of K stages starting at stage s0 reads the skewed block of stages
    // 32*(s0/32).., offset by d = s0 % 32 stages: its time step t is block row
    // t + 2d and its stage k is block column k + d.
    auto block = [&](int s) {
        return skew + (skOff[(size_t)(m0 * 2 + c) * nq + (s >> 5)] + 2 * (s & 31)) * 32;
    };
    if (live) {
        while (S - s0 >= KMAX && n > 0) {
            sweep_pass<T, KMAX>(chain, ldc, n, block(s0), s0 & 31);
            n -= KMAX;
            s0 += KMAX;
        }
    }
    // remaining stages: 16, 8, 4, 2, 1
#define HPX_SUBPASS(KK)                                                                   \
    if (KK < KMAX && live && S - s0 >= KK && n > 0) {                                     \
        sweep_pass<T, KK>(chain, ldc, n, block(s0), s0 & 31);                            \
        n -= KK;                                                                          \
        s0 += KK;                                                                         \
    }
    HPX_SUBPASS(16)
    HPX_SUBPASS(8)
    HPX_SUBPASS(4)
    HPX_SUBPASS(2)
    HPX_SUBPASS(1)
#undef HPX_SUBPASS
    if (!live) return;
    // n == chain_len(m, c, L): degrees l = m + c + 2i
    cplx<T>* out = alm + (int64_t)col * nalm;
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2 + m + c;
    for (int i = 0; i < n; ++i) out[base + 2 * i] = chain[(int64_t)i * ldc];
}

// Small batches (fewer than 16 maps) leave most lanes of the kernel above idle;
// they use this layout instead: one warp per parity chain, lane s applies stage
// s of a pass of 32 sweeps, the chain streams through the lanes as a wavefront
// (lane s two steps behind lane s-1, values handed on by warp shuffles), G maps
// per lane share each angle load.
template <class T, int G>
__global__ void __launch_bounds__(64) rot_stage_kernel(const cplx<T>* __restrict__ beta, cplx<T>* __restrict__ alm,
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
            if (b0 + g < B) v = beta[(((int64_t)m * 2 + par) * P2 + q) * B + (b0 + g)];
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
    // one lane per map: from 16 maps (FP64) or 4 maps (FP32, whose angle rows are
    // staged ahead by cp.async: at nside 2048 the per-stage angle tables of
    // rot_stage_kernel, 134 MB, no longer stay in L2 and its per-step loads wait
    // on DRAM)
    if (g.B >= (sizeof(T) == 4 ? 4 : 16)) {
        const int ngroups = (g.B + 31) / 32;
        const int nitems = (g.L + 1) * 2 * ngroups;
        const int threads = 64;
        const int blocks = (nitems * 32 + threads - 1) / threads;
        if constexpr (sizeof(T) == 4) {
            // the plan's form (HPX_FLAG_AUTOTUNE): one complex column per lane with 32
            // stages per pass (168 registers, 12 warps per SM) or 16 (twice the passes
            // over the chains, 20 warps per SM), or one real column per lane with 32
            // stages (128 registers, 16 warps per SM, 2B lanes for B maps)
            if (P->rotForm == 2) {   // one real column per lane
                const int rgroups = (2 * g.B + 31) / 32, ritems = (g.L + 1) * 2 * rgroups;
                rot_staged_real_kernel<32><<<(ritems * 32 + threads - 1) / threads, threads, 0, s>>>(
                    (cplx<float>*)P->beta, (cplx<float>*)alm, P->t.skOff, (const cplx<float>*)P->t.skew, P->t.nq,
                    g.P2, g.L, g.B, g.nalm, rgroups, ritems);
            } else if (P->rotForm == 1)
                rot_staged_kernel<16><<<blocks, threads, 0, s>>>((cplx<float>*)P->beta, (cplx<float>*)alm,
                                                                P->t.skOff, (const cplx<float>*)P->t.skew, P->t.nq,
                                                                g.P2, g.L, g.B, g.nalm, ngroups, nitems);
            else
                rot_staged_kernel<32><<<blocks, threads, 0, s>>>((cplx<float>*)P->beta, (cplx<float>*)alm,
                                                                P->t.skOff, (const cplx<float>*)P->t.skew, P->t.nq,
                                                                g.P2, g.L, g.B, g.nalm, ngroups, nitems);
        } else {
            rot_kernel<T, 16><<<blocks, threads, 0, s>>>((cplx<T>*)P->beta, (cplx<T>*)alm, P->t.skOff,
                                                        (const cplx<T>*)P->t.skew, P->t.nq, g.P2, g.L, g.B,
                                                        g.nalm, ngroups, nitems);
        }
        return;
    }
    const int nmax = g.L / 2 + 1;
    constexpr int G = 1;
    const size_t smem = (size_t)2 * nmax * 2 * G * sizeof(T);
    cudaFuncSetAttribute(rot_stage_kernel<T, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid(g.L + 1, g.B);
    rot_stage_kernel<T, G><<<grid, 64, smem, s>>>((const cplx<T>*)P->beta, (cplx<T>*)alm, P->t.angOff,
                                                  (const cplx<T>*)P->t.ang, g.p, g.P2, g.L, g.B, g.nalm, nmax);
}

template void launch_rot<float>(const hpx_plan_s*, float*, cudaStream_t);
template void launch_rot<double>(const hpx_plan_s*, double*, cudaStream_t);

}  // namespace hpx
