// Internal plan object of the HP2SPH library and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "../../include/hpx.h"
#include "common.cuh"

struct hpx_plan_s;

namespace hpx {

// Device copies of the set-up tables (element type T = plan precision where
// marked "T"; FP64-built on the host and rounded once).
struct DevTables {
    int *nphi = nullptr, *startN = nullptr, *startS = nullptr, *pow2 = nullptr, *logn = nullptr,
        *fftL = nullptr, *logL = nullptr;
    int64_t *shOff = nullptr, *chOff = nullptr, *bhOff = nullptr;
    void *shift = nullptr, *chirp = nullptr, *bhat = nullptr, *twid = nullptr;   // cplx<T>
    int64_t *ch4Off = nullptr, *bh4Off = nullptr;   // quarter-length Bluestein tables (ring form 1)
    void *chirp4 = nullptr, *bhat4 = nullptr;       // cplx<T>
    int *poleN = nullptr, *poleS = nullptr;
    double* polew = nullptr;
    int npole = 0;
    int *rowptr = nullptr, *ent = nullptr;
    void *entw = nullptr, *dec = nullptr;   // T
    int* nstart = nullptr;                  // dense spreading table: first node per grid point
    void* swts = nullptr;                   // T [spreadE][M]
    int spreadE = 0;
    int* tstart = nullptr;                  // interpolation (transpose of the half-grid spreading)
    void* hwn = nullptr;                    // T [interpE][Q][2]
    int interpE = 0, interpRows = 0, interpD = 0;
    int* hstart = nullptr;                  // half-grid spreading with folded mirrors
    void* hwts = nullptr;                   // T [spreadH][M/2 + 1][2]
    int spreadH = 0, spreadRows = 0, spreadD = 0;
    void* D = nullptr;                      // T [2][2][P2][P2]
    void* C = nullptr;                      // T [2][2][P2][P2]: change of basis alone (HPX_FLAG_CG)
    void* cgH = nullptr;                    // cplx<T> [4][2][cgN]: CG matrix-vector tables
    int cgN = 0, cgk0[4] = {0, 0, 0, 0}, cgn[4] = {0, 0, 0, 0};
    void* Es = nullptr;                     // T [2][2][P2][P2]: Legendre-0/1 -> latitude Fourier (synthesis)
    int* shifted = nullptr;                 // per ring pair: first pixel at pi / nphi (1) or 0 (0)
    int64_t* angOff = nullptr;
    void* ang = nullptr;                    // cplx<T> (cos, sin)
    int64_t* skOff = nullptr;               // skewed angle blocks for the sweep wavefront
    void* skew = nullptr;                   // cplx<T>
    int nq = 0;
    void* skewT = nullptr;                  // cplx<T>, transposed sweeps
    int *nrowptr = nullptr, *nent = nullptr;   // NUFFT transpose: CSR over nodes
    void* nentw = nullptr;                  // T
};

struct Geometry {
    int ns, p, L, Q, npairs, M, P2, Lmax, smem_ring, B;
    int64_t npix, nalm;
};

}  // namespace hpx

struct hpx_plan_s {
    hpx::Geometry g;
    int precision;
    int device;
    cudaStream_t stream;
    hpx::DevTables t;
    // workspace
    void* Y = nullptr;      // cplx<T> [B][Q][p+1]: step-1 ring coefficients per latitude node
    void* U = nullptr;      // cplx<T> [B][L+1][ldu]: spread half grids (t = 0..M/2) per column
    int ldu = 0;
    void* bvec = nullptr;   // cplx<T> [B][p+1][2][P2]: latitude NUFFT right-hand sides
    void* beta = nullptr;   // cplx<T> [B][p+1][2][P2]: order-0/1 Legendre coefficients (aliases Y)
    int64_t bytes = 0;
    int status = 0;
    // ring FFT launches by transform length (pow2 rings: nphi; others: the
    // Bluestein length): ring pairs ringList[first .. first + count - 1]
    struct RingClass {
        int N, first, count;
        bool blue;   // N >= kRingCtMin: every ring of the class is a Bluestein ring (else none is)
    };
    std::vector<RingClass> ringClasses;
    int* ringList = nullptr;
    // profiling: events around the kernels of each recorded hpx_analyze call
    static constexpr int kMaxProf = 256;
    static constexpr int kStages = 6;
    bool prof = false;
    int nprof = 0;
    cudaEvent_t* ev = nullptr;   // [kMaxProf][kStages + 1]
    // per-order operators M_{m,c} (default analysis path; see k_fused.cu)
    unsigned flags = 0;
    void* fusedM = nullptr;        // T, n_alm x P2
    int64_t* fusedOff = nullptr;   // first row of (m, c)
    int* fusedTiles = nullptr;     // (m, c, first row) per block of the apply kernel
    int fused_ntiles = 0;
    int fused_ldm = 0;             // row stride of M (P2 rounded up to a multiple of 4)
    bool use_tc = false;           // FP32: apply M with tcgen05 MMAs (k_fused_tc.cu)
    // tensor-core layout of M (use_tc): tile t (128 rows of one chain, rows
    // padded to a multiple of 8 = rp) is stored as consecutive K-chunks of
    // rp x 128 bytes in the MMA's core-matrix order, from 4-byte offset tcOff[t]
    // (rp x 32 floats, or after prepare_fused_tc the FP16 pairs of the scaled rows)
    int64_t* tcOff = nullptr;
    int* tcFirst = nullptr;        // first tile of (m, c)
    float* tcRinv = nullptr;       // FP16 form: 1 / row scale, per stored row of the tiles
    float* bscale = nullptr;       // FP16 form: [B][L+1] largest magnitude of each b column
    unsigned char* bpk = nullptr;  // FP16 form: b as scaled FP16 pairs in the MMA layout (fp16pair.cuh)
    int* d_status = nullptr;       // device status word (timed-out waits, non-finite inputs)
    int64_t fused_bytes = 0;       // bytes of M
    void* synM = nullptr;          // T, n_alm x ldm row-major: synthesis operators R_{m,c} Es (HPX_FLAG_SYNTHESIS)
    // FP32 plans on the tensor cores: the synthesis operators transposed into
    // tiles of 128 latitude modes x the chain's degrees (FP16 pairs, K-chunks of
    // 32), their row scales, the tile table (m, c, k0), each tile's K-chunk count,
    // operator offset and first row scale; the packed coefficients and their
    // per-(map, m, c) scales
    void* synT = nullptr;
    void* synRinv = nullptr;
    int* synTiles = nullptr;
    int* synNch = nullptr;
    int64_t* synOff = nullptr;
    int64_t* synRowBase = nullptr;
    void* synScale = nullptr;
    void* synBpk = nullptr;
    int synNtiles = 0;
    void* jres = nullptr;          // T [B][npix]: Jacobi residual maps (HPX_FLAG_JACOBI)
    void* jalm = nullptr;          // cplx<T> [B][n_alm]: Jacobi update
    // sub-plan of an uneven batch whose maps are not adjacent in the caller's
    // array: element offset of each of its maps there (read by the ring and pole
    // stages of the analysis, which then take the caller's base pointer)
    int64_t* mapIdx = nullptr;
    // sweeps path of FP32 plans of 4 maps or more, nside <= 1024: D on the tensor cores
    // (prepare_dense_tc): its distinct tiles in the FP16-pair form, 1 / row scale,
    // and the CTA tiles (m, par, first row) with their operator offsets
    void* dTC = nullptr;
    void* dRinv = nullptr;
    int* dTiles = nullptr;
    int64_t* dTcOff = nullptr;
    int dNtiles = 0;
    float tuned_ms[2] = {0.f, 0.f};   // HPX_FLAG_AUTOTUNE: ms per analysis, operators / sweeps
    // launch shapes of the compile-time FFT kernels: elements per thread (16 or 32)
    // of the ring stage and of the grid FFT (HPX_FLAG_AUTOTUNE times both)
    int ringE = 16, latE = 16;
    // Bluestein ring classes of 4096 points and more: one convolution of the whole
    // ring (0) or four of its quarter-length subsequences (1; HPX_FLAG_AUTOTUNE)
    int ringForm = 0;
    // form of the FP32 run-time sweeps (HPX_FLAG_AUTOTUNE): 0 = one complex column
    // per lane, 32 stages per pass; 1 = the same with 16 stages; 2 = one real
    // column per lane, 32 stages
    int rotForm = 0;
    // the tensor-core paths' packed b: written by the grid-FFT kernel (0) or by
    // a separate full-line pass over FP32 b (1; HPX_FLAG_AUTOTUNE)
    int packSep = 0;

    // uneven batches (group plans): one uniform sub-plan per distinct nside
    bool group = false;
    std::vector<hpx_plan_s*> subs;
    std::vector<int> sub_count, sub_first;   // maps per sub-plan, first entry in d_idx
    std::vector<int> sub_inplace;            // 1: the sub-plan's maps are adjacent in the batch
    std::vector<int64_t> sub_mapoff, sub_almoff, sub_cloff;   // byte offsets of an in-place run
    int* d_idx = nullptr;                    // batch index of every map, grouped by sub-plan
    int64_t* d_mapoff = nullptr;             // byte offset of map i in the caller's arrays
    int64_t* d_almoff = nullptr;
    int64_t* d_cloff = nullptr;
    int64_t* d_almel = nullptr;              // element offsets of map i's coefficients / spectrum
    int64_t* d_clel = nullptr;
    int* d_lmax = nullptr;                   // lmax of map i
    std::vector<void*> stage_maps, stage_alm, stage_cl;   // per sub-plan staging (gathered runs)
    std::vector<cudaStream_t> sstreams;      // per sub-plan stream (concurrent branches of an analysis)
    std::vector<cudaEvent_t> sjoin;          // per sub-plan join event
    cudaEvent_t sfork = nullptr;             // fork event on the group's stream
    void* ringJobs = nullptr;                // RingJob<T> per sub-plan (persistent ring kernel)
    int4* ringItems = nullptr;               // (sub-plan, ring pair, map, length), longest first
    int nRingItems = 0, nRingLong = 0;   // items, of which the first nRingLong have 1024 or 2048 points
    cudaEvent_t ringEv = nullptr;        // recorded after the short-ring launches
    int64_t total_npix = 0, total_nalm = 0, total_ncl = 0;

    // CUDA graphs of hpx_analyze (HPX_FLAG_GRAPH)
    cudaStream_t cap = nullptr;
    struct GraphEntry {
        const void* maps;
        void* alm;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;
};

namespace hpx {

// One sub-plan of an uneven batch as seen by the persistent ring kernel: its
// tables and Y workspace, and where its maps are (staged: a plan-owned staging
// buffer; else the caller's array plus mapoff elements).
template <class T>
struct RingJob {
    int64_t mapoff;            // element offset of the sub-plan's first map (adjacent maps)
    const int64_t* mapIdx;     // else: element offset of each of its maps
    cplx<T>* Y;
    const int *nphi, *startN, *startS, *pow2, *logn, *fftL, *logL, *shifted;
    const int64_t *shOff, *chOff, *bhOff;
    const cplx<T> *shift, *chirp, *bhat, *tw;
    int twlen, p, Q, L;
    int64_t npix;
};
template <class T>
void launch_ring_list(const RingJob<T>* jobs, const int4* items, int nitems, int nlong, const T* maps_base,
                      cudaStream_t s);

// ring transforms of this many points or more run in launches of one length and
// one kind (plain or Bluestein) with the compile-time FFT of fft_ct.cuh
constexpr int kRingCtMin = 4096;

// ew != 0: the rows of the equal-weight quadrature's ring stage (every m <= lmax,
// aliased mod nphi, synthesis fold weights, times ew) instead of the analysis'
// ring classes of minN points or more only (minN > 0: the rest ran elsewhere)
template <class T> void launch_ring_fft(const hpx_plan_s* P, const T* maps, cudaStream_t s, T ew = T(0), int minN = 0);
template <class T> void launch_poles(const hpx_plan_s* P, const T* maps, cudaStream_t s);
template <class T> void launch_nufft(const hpx_plan_s* P, cudaStream_t s);
template <class T> void launch_spread(const hpx_plan_s* P, cudaStream_t s);
// packed: also (FP32 tensor-core plans) write b as the FP16 pairs of bpk, with
// each column's largest magnitude in bscale, instead of bvec
template <class T> void launch_lat_fft(const hpx_plan_s* P, cudaStream_t s, bool packed = false);
// whether the analysis' contraction reads the packed b (bpk) of this plan
bool packs_b(const hpx_plan_s* P);

template <class T> void launch_dense(const hpx_plan_s* P, cudaStream_t s, const void* Dmat = nullptr);
template <class T> void launch_cg(const hpx_plan_s* P, cudaStream_t s);
template <class T> void launch_rot(const hpx_plan_s* P, T* alm, cudaStream_t s);
int fused_tile_rows(int B);
// per-order operators on the FP32 pipes; Mrows: row-major operators of the
// layout of fusedM's SIMT form (NULL = fusedM), e.g. the synthesis operators synM
template <class T> void launch_fused(const hpx_plan_s* P, T* alm, cudaStream_t s, const void* Mrows = nullptr);
// S^T of the spherical-harmonic synthesis times `scale` (maps -> alm) and the
// Jacobi-refined equal-weight analysis of the HEALPix software (k_healpix.cu)
template <class T> void launch_sh_adjoint(const hpx_plan_s* P, const T* maps, T* alm, cudaStream_t s, T scale);
template <class T> void launch_healpix_jacobi(const hpx_plan_s* P, const T* maps, T* alm, int niter, cudaStream_t s);
void launch_fused_tc(const hpx_plan_s* P, float* alm, cudaStream_t s);
// after build_fused<float> of the tensor-core layout: converts M to the form
// launch_fused_tc reads (and allocates its scale arrays); 0 on success
int prepare_fused_tc(hpx_plan_s* P);
// D of the sweeps path on the tensor cores: plan-time layout (0 on success) and
// the launch (bvec -> beta, like launch_dense)
int prepare_dense_tc(hpx_plan_s* P);
// the synthesis operators on the tensor cores (from synM; 0 on success) and the
// launch (alm -> bvec, like launch_synth_apply)
int prepare_synth_tc(hpx_plan_s* P);
void launch_synth_tc(const hpx_plan_s* P, const float* alm, cudaStream_t s);
void launch_dense_tc(const hpx_plan_s* P, cudaStream_t s);
void launch_timeout_selftest(const hpx_plan_s* P, int spins, cudaStream_t s);
// HPX_FLAG_CHECKED: records HPX_ERR_NONFINITE in *status if any of the n reals
// (float or double) at x is NaN or infinite.
void launch_finite_check(const void* x, int64_t n, bool fp64, int* status, cudaStream_t s);
template <class T>
int build_fused(hpx_plan_s* P, const double* D64, const cplx<double>* skew64, cudaStream_t s, void* out, bool tiled);
template <class T> void launch_synth_apply(const hpx_plan_s* P, const T* alm, cudaStream_t s);
// float offset of element (row r of a tile with rp rows, column k) in the
// tensor-core layout of M, relative to the tile's first chunk
__host__ __device__ inline int64_t tc_elem(int rp, int r, int k) {
    return (int64_t)(k >> 5) * rp * 32 + (r >> 3) * 256 + ((k & 31) >> 2) * 32 + (r & 7) * 4 + (k & 3);
}
// transpose of the analysis; wpos = weight of the m > 0 coefficients (2: the
// adjoint under the real-map inner product, 1: under the plain Euclidean one)
// type-2 latitude NUFFT of the adjoint and the synthesis in two kernels
// (k_nufft2.cu); false where they do not apply (then nufft_adj_kernel runs)
bool launch_nufft2(const hpx_plan_s* P, cudaStream_t s);
template <class T> void launch_adjoint(const hpx_plan_s* P, const T* alm, T* maps, cudaStream_t s, T wpos = T(2));
// ev: NULL, or kStages + 1 events recorded around its stages (profiling)
template <class T>
void launch_sh_synthesis(const hpx_plan_s* P, const T* alm, T* maps, cudaStream_t s, cudaEvent_t* ev = nullptr);
int group_sh_synthesis(hpx_plan_s* P, const void* alm, void* maps);
// uneven batches (group.cu)
hpx_plan_s* group_create(const hpx_plan_desc* d, int* err);
int group_analyze(hpx_plan_s* P, const void* maps, void* alm);
int group_synthesize(hpx_plan_s* P, const void* alm, void* maps);
int group_cl(hpx_plan_s* P, const void* alm, double* cl);
int group_analyze_vjp(hpx_plan_s* P, const void* galm, void* gmaps);
bool group_build_ring_list(hpx_plan_s* G);
// the analysis of a uniform plan without its ring stage (Y already holds the
// ring coefficients): poles onward (capi.cu)
int analyze_after_rings(hpx_plan_s* P, const void* maps, void* alm);
void group_free(hpx_plan_s* P);
template <class T> void launch_cl(const hpx_plan_s* P, const T* alm, double* cl, cudaStream_t s);
// dL/da of Eq. (APS) for gcl = dL/dC (k_cl.cu); almoff / cloff / lmax: per-map
// element offsets and degrees (NULL for a uniform batch: b nalm_u, b (Lu + 1), Lu)
template <class T>
void launch_cl_vjp(const T* alm, const double* gcl, T* galm, const int64_t* almoff, const int64_t* cloff,
                   const int* lmax, int Lmax_all, int B, int Lu, int64_t nalm_u, cudaStream_t s);

}  // namespace hpx
