/*
 * hpx.h -- C ABI of the GB300 HP2SPH library: spherical-harmonic analysis of
 * real HEALPix maps by the method of Drake & Wright, "A Fast and Accurate
 * Algorithm for Spherical Harmonic Analysis on HEALPix Grids" (arXiv:1904.10514),
 * Algorithm 1, and the angular power spectrum C_l of Eq. (APS).
 *
 * All pointers to map, coefficient and spectrum buffers are DEVICE pointers
 * (cudaMalloc'd, or torch tensors on the plan's device), contiguous, and owned
 * by the caller.  The plan owns every table and workspace it needs; no call
 * allocates device memory after hpx_plan / hpx_plan_ex has returned.  Calls are
 * asynchronous on the plan's stream (hpx_set_stream); hpx_sync waits.
 *
 * Layouts
 *   maps : [batch][12 * nside^2] real, RING order (north to south, increasing
 *          longitude within a ring), element type = plan precision
 *          (float for HPX_FP32, double for HPX_FP64).
 *   alm  : [batch][n_alm][2] (re, im) of the plan precision, m >= 0 only,
 *          packed m-major: idx(l, m) = m (2 lmax + 1 - m) / 2 + l,
 *          n_alm = (lmax + 1)(lmax + 2) / 2.  For a real map
 *          a_l^{-m} = (-1)^m conj(a_l^m) (Appendix A conventions: orthonormal
 *          Y_l^m with the Condon-Shortley phase).
 *   cl   : [batch][lmax + 1] double.
 *
 * Method parameters: p = 2 nside latitude/longitude half-bandwidth, lmax <= p
 * (Sec. 3.2.2 / 3.3: the method yields degrees up to p); nside must be a power
 * of two, 2 <= nside <= 2048 (FP64 plans: nside <= 1024): the shared-memory
 * FFT and NUFFT grids of one ring / one column must fit in one thread block.
 *
 * Return codes: 0 on success, a negative HPX_ERR_* otherwise; hpx_last_error()
 * gives the last code of the calling thread and hpx_strerror() a message.  No
 * C++ exception crosses this interface.
 */
#ifndef HPX_H
#define HPX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HPX_OK 0
#define HPX_ERR_ARG -1      /* null pointer or inconsistent argument              */
#define HPX_ERR_NSIDE -2    /* nside not a power of two in the supported range   */
#define HPX_ERR_LMAX -3     /* lmax < 0 or lmax > 2 nside                         */
#define HPX_ERR_CUDA -4     /* a CUDA runtime call failed                         */
#define HPX_ERR_OOM -5      /* device memory for tables / workspace not available */
#define HPX_ERR_TIMEOUT -6  /* a bounded device-side wait gave up                 */
#define HPX_ERR_STATE -7    /* call not valid for this plan                       */
#define HPX_ERR_NONFINITE -8 /* HPX_FLAG_CHECKED: an input held NaN or infinity   */

#define HPX_FP32 0
#define HPX_FP64 1

/* Plan flags.
 * HPX_FLAG_SWEEPS: apply the latitude operator D and the Givens sweeps of the
 *   Fourier-to-SH conversion at run time (two kernels per call).  Without it the
 *   plan composes, for every order m and parity chain, D with the sweeps into
 *   one matrix M_{m,c} (built once in FP64 on the GPU from the same rotations,
 *   n_alm x (nside + 1) entries, 8.6 GB in FP32 at nside 1024) and the analysis
 *   applies those as one batched contraction; if that memory is not available,
 *   or the operators would exceed 24 GB (nside 2048 needs 69 GB and minutes of
 *   FP64 build), the plan uses the sweeps and sets this flag (hpx_plan_flags).
 *   With the sweeps, FP32 plans of 4 maps or more and nside <= 1024 apply D on
 *   the tensor cores (the FP16-pair arithmetic of the operators, D resident in
 *   L2), unless HPX_FLAG_SIMT or HPX_FLAG_CG is given. */
#define HPX_FLAG_SWEEPS 1u
/* HPX_FLAG_GRAPH: the first hpx_analyze call with a given (maps, alm) pair
 *   captures the plan's whole launch sequence into a CUDA graph (on a stream of
 *   the plan's own); later calls with the same pair replay it with one graph
 *   launch on the plan's stream.  Must not be used while the caller is itself
 *   capturing the plan's stream. */
#define HPX_FLAG_GRAPH 2u
/* HPX_FLAG_SIMT: apply the per-order operators of an FP32 plan on the FP32
 *   pipes.  By default FP32 plans of 9 or more maps use the tensor cores
 *   (tcgen05: each operand, scaled by a power of two, split into a pair of
 *   FP16 numbers, three kind::f16 MMAs accumulated in FP32; the relative error
 *   of each product is below 2^-22, as with FP32 rounding). */
#define HPX_FLAG_SIMT 4u
/* HPX_FLAG_CHECKED: every hpx_analyze / hpx_synthesize first checks on the host
 *   that its two pointers are device (or managed) memory of the plan's device
 *   (else HPX_ERR_ARG, nothing is launched), and on the device that the input
 *   holds only finite values (else HPX_ERR_NONFINITE is recorded in the plan's
 *   status word and reported by the next hpx_sync; the outputs are then
 *   undefined).  Costs one extra read of the input. */
#define HPX_FLAG_CHECKED 8u
/* HPX_FLAG_AUTOTUNE: at plan creation, on scratch buffers allocated and freed
 *   inside hpx_plan_ex: (1) time the ring-FFT and grid-FFT stages of the plan's
 *   batch with 16 and with 32 elements per thread (launch shapes of the
 *   compile-time FFT kernels), for FP32 plans that run the sweeps per call the
 *   three forms of the sweep kernel, for the tensor-core paths the two
 *   placements of the packing of b, and the two forms of the Bluestein ring
 *   classes of 4096 points and more, and keep the fastest of each
 *   (hpx_plan_tuning; remembered per nside, lmax, batch, precision and path for
 *   the process's later plans); (2) when the
 *   per-order operators were built, time one analysis
 *   through them and through the run-time sweeps and keep the faster path; if
 *   that is the sweeps the operators are freed and HPX_FLAG_SWEEPS is set
 *   (hpx_plan_flags). */
#define HPX_FLAG_AUTOTUNE 16u
/* HPX_FLAG_SYNTHESIS: also build the table of hpx_sh_synthesis (the expansion
 *   of the order-0/1 Legendre functions in the latitude Fourier basis, FP64 on
 *   the host at plan time, 4 (nside + 1)^2 entries). */
#define HPX_FLAG_SYNTHESIS 32u
/* HPX_FLAG_CG: solve the latitude least squares of every column by conjugate
 *   gradients on its normal equations (Sec. 3.2.2; matrix-vector products by
 *   FFT of the Toeplitz-plus-Hankel Gram matrix), then apply the change of basis
 *   to order-0/1 Legendre functions and the Givens sweeps at run time.  The form
 *   the paper describes, kept as an ablation of the default premultiplied
 *   operators; implies HPX_FLAG_SWEEPS.  Stops at a relative residual of 1e-7
 *   (FP32) or 1e-14 (FP64). */
#define HPX_FLAG_CG 64u
/* HPX_FLAG_JACOBI: also allocate the workspace of hpx_healpix_analysis (one map
 *   buffer and one coefficient buffer of the batch); implies HPX_FLAG_SYNTHESIS.
 *   Uniform plans only (else HPX_ERR_ARG). */
#define HPX_FLAG_JACOBI 128u

typedef struct hpx_plan_s hpx_plan_s;

typedef struct hpx_plan_desc {
    int nside;        /* HEALPix resolution parameter N_side (power of two)       */
    int lmax;         /* largest degree returned, 0 <= lmax <= 2 nside; -1 = 2 nside */
    int batch;        /* number of maps processed per call, >= 1                  */
    int precision;    /* HPX_FP32 or HPX_FP64                                     */
    unsigned flags;   /* HPX_FLAG_* (SWEEPS, GRAPH, SIMT, CHECKED, AUTOTUNE, SYNTHESIS, CG, JACOBI), or 0 */
    /* Uneven batches: NULL, or `batch` values giving the nside of every map
     * (then `nside` is ignored).  Maps, coefficients and spectra are then
     * concatenated in the given order: map i occupies 12 nside_i^2 elements of
     * `maps`, n_alm(lmax_i) coefficients of `alm` and lmax_i + 1 values of `cl`,
     * with lmax_i = 2 nside_i when lmax = -1, else lmax (<= 2 min nside_i).  The
     * plan holds one uniform sub-plan per distinct (nside, lmax); maps of one
     * sub-plan that are adjacent in the batch are used in place, others are
     * gathered into plan-owned staging buffers.  The caller's array must
     * outlive the call. */
    const int* nsides;
    /* Per-map degrees: NULL, or `batch` values lmax_i (-1 = 2 nside_i, else
     * 0 <= lmax_i <= 2 nside_i) overriding `lmax`; the layouts are then
     * concatenated as for `nsides` (with n_alm(lmax_i) and lmax_i + 1 entries per
     * map), also when `nsides` is NULL (every map then has `nside`). */
    const int* lmaxs;
} hpx_plan_desc;

/* Plan for `batch` real FP32 maps of one nside on the current CUDA device
 * (Algorithm 1, all steps).  Builds the FP64 set-up tables (ring geometry of
 * Eq. healpts, FFT chirps and shifts of Sec. 3.1, pole-fit weights of
 * Sec. 3.2.1, NUFFT spreading tables and the latitude least-squares operator of
 * Sec. 3.2.2, the Givens rotation angles of Sec. 3.3) and allocates the
 * workspace.  Returns NULL on error (see hpx_last_error). */
hpx_plan_s* hpx_plan(int nside, int lmax, int batch);

/* Same, with precision and flags from a descriptor.  NULL on error. */
hpx_plan_s* hpx_plan_ex(const hpx_plan_desc* desc);

/* Stream for the plan's launches (a cudaStream_t); NULL = legacy stream. */
int hpx_set_stream(hpx_plan_s* plan, void* cuda_stream);

/* HP2SPH analysis (Algorithm 1): maps -> alm, layouts above.  Asynchronous. */
int hpx_analyze(hpx_plan_s* plan, const void* maps, void* alm);

/* The exact adjoint (transpose) of hpx_analyze with respect to the real inner
 * products <f, g> = sum_i f_i g_i on maps and
 * <a, b> = sum_l [Re(a_l0 conj b_l0) + 2 sum_{m>0} Re(a_lm conj b_lm)] on alm:
 * alm -> maps.  It is not the spherical-harmonic synthesis.  The imaginary part
 * of an input a_l0 is ignored (the analysis always returns a real a_l0).
 * Asynchronous. */
int hpx_synthesize(hpx_plan_s* plan, const void* alm, void* maps);

/* Spherical-harmonic synthesis of real maps (the direction the paper names as
 * future work; Appendix A conventions):
 *     f(theta_p, phi_p) = sum_{l <= lmax} sum_{|m| <= l} a_l^m Y_l^m(theta_p, phi_p)
 * at every pixel centre, with a_l^{-m} = (-1)^m conj(a_l^m) and the imaginary
 * part of a_l0 ignored.  alm -> maps in the layouts above.  Exact up to rounding
 * and the NUFFT accuracy for any coefficients (it is not the inverse of
 * hpx_analyze, which is a least-squares approximation).  The orders are
 * converted to order 0/1 by the transposed Givens sweeps (Sec. 3.3), expanded in
 * cos/sin(j theta), evaluated at the ring latitudes by a type-2 NUFFT and folded
 * into each ring's nphi frequencies before an inverse FFT per ring.  Requires a
 * plan made with HPX_FLAG_SYNTHESIS (else HPX_ERR_STATE).  Asynchronous. */
int hpx_sh_synthesis(hpx_plan_s* plan, const void* alm, void* maps);

/* Vector-Jacobian product of hpx_analyze, for gradients of a loss L(alm) with
 * respect to the maps.  galm = dL/dRe(a) + i dL/dIm(a) for every stored
 * coefficient (the packed m >= 0 array read as independent real and imaginary
 * parts, the convention torch uses for complex tensors); gmaps = dL/df, i.e.
 * gmaps_i = sum over stored (l, m) of Re(conj(galm_lm) d a_lm / d f_i).  It is
 * the transpose of the analysis (Algorithm 1 step by step, in reverse) under
 * the plain Euclidean inner product on the packed array: hpx_synthesize with
 * unit instead of doubled weight on m > 0.  The imaginary parts of galm at
 * m = 0 and m = 2 nside are ignored (the analysis returns those coefficients
 * real).  Layouts as hpx_synthesize (uneven batches concatenated); gmaps is
 * overwritten.  Asynchronous. */
int hpx_analyze_vjp(hpx_plan_s* plan, const void* galm, void* gmaps);

/* Vector-Jacobian product of hpx_cl (Eq. APS): given gcl = dL/dC_l
 * ([batch][lmax + 1] double, device) and the coefficients alm the spectrum was
 * computed from, writes galm = dL/dRe(a) + i dL/dIm(a) in alm's layout and
 * precision:  galm_lm = gcl_l * 2 w_m a_lm / (2l + 1), w_0 = 1, w_m = 2 (m > 0).
 * Uneven batches: alm, gcl and galm concatenated as for hpx_cl.  galm may not
 * alias alm.  Asynchronous. */
int hpx_cl_vjp(hpx_plan_s* plan, const void* alm, const double* gcl, void* galm);

/* The transpose of hpx_sh_synthesis with respect to the library's real inner
 * products (maps: sum_i f_i g_i; coefficients: weight 2 for m > 0):
 *     alm_l^m = sum_i conj(Y_l^m(x_i)) f(x_i),   m >= 0,
 * the unweighted pixel sum of Eq. (healsph) (Sec. 2.2).  maps -> alm in the
 * plan's layouts; requires a uniform plan made with HPX_FLAG_SYNTHESIS (else
 * HPX_ERR_STATE).  Asynchronous. */
int hpx_sh_synthesis_adjoint(hpx_plan_s* plan, const void* maps, void* alm);

/* The analysis of the HEALPix software that the paper compares HP2SPH with
 * (Sec. 2.2): the equal-weight quadrature of Eq. (healsph),
 * a = (4 pi / N) S^* f, followed by `niter` steps of the Jacobi (Richardson)
 * iteration of Eqs. (uzawa) / (richardson), a <- a + (4 pi / N) S^* (f - S a),
 * S = hpx_sh_synthesis (the software's default is niter = 3).  maps -> alm in the
 * plan's layouts; requires a plan made with HPX_FLAG_JACOBI (else
 * HPX_ERR_STATE); 0 <= niter <= 1000.  Asynchronous. */
int hpx_healpix_analysis(hpx_plan_s* plan, const void* maps, void* alm, int niter);

/* Angular power spectrum of Eq. (APS) for real maps,
 * C_l = (|a_l0|^2 + 2 sum_{m=1}^{l} |a_lm|^2) / (2l + 1),
 * squares summed in groups of 4 in the plan precision, the group sums in
 * double, partial sums combined with compensated summation (all terms are
 * positive; the result is within about 3e-7 relative for FP32 plans and
 * 1e-13 for FP64 plans).  alm in the plan's layout
 * and precision, cl = [batch][lmax + 1] double (device).  Asynchronous. */
int hpx_cl(hpx_plan_s* plan, const void* alm, double* cl);

/* Wait for the plan's stream; returns the first asynchronous error. */
int hpx_sync(hpx_plan_s* plan);

/* Release the plan's tables and workspace (waits for its stream). */
void hpx_destroy(hpx_plan_s* plan);

/* Sizes of the plan's layouts (0 for a NULL plan). */
int64_t hpx_npix(const hpx_plan_s* plan);
int64_t hpx_nalm(const hpx_plan_s* plan);
int hpx_plan_lmax(const hpx_plan_s* plan);
/* Bytes of device memory the plan holds (tables + workspace). */
int64_t hpx_plan_bytes(const hpx_plan_s* plan);
/* Flags in effect (HPX_FLAG_SWEEPS set when the sweeps run at call time). */
int hpx_plan_flags(const hpx_plan_s* plan);
/* Kernel launches of one hpx_analyze call (ring FFTs: one per transform length). */
int hpx_plan_launches(const hpx_plan_s* plan);
/* Launch shapes in effect (HPX_FLAG_AUTOTUNE, else 16, 16, 0, 0 and 0):
 * elements per thread of the ring-FFT and of the grid-FFT kernels, the form of
 * the FP32 run-time Givens sweeps of 4 maps or more (0: one complex column per
 * lane, 32 stages per pass; 1: the same with 16 stages; 2: one real column per
 * lane, 32 stages), whether the tensor-core paths' FP16-pair right-hand sides
 * are written by a pass of their own (1) or by the grid-FFT kernel (0), and the
 * form of the Bluestein ring classes of 4096 points and more (0: one
 * convolution of the whole ring; 1: the DFT of nphi = 4j points from four
 * Bluestein transforms of its quarter-length subsequences and one radix-4 step).
 * HPX_ERR_ARG for NULL arguments or an uneven-batch plan. */
int hpx_plan_tuning(const hpx_plan_s* plan, int* ring_elems, int* fft_elems, int* sweep_form, int* pack_pass,
                    int* ring_form);
/* Sets those launch shapes (16 or 32, 16 or 32, 0..2, 0 or 1, 0 or 1; e.g. the
 * values an earlier process's HPX_FLAG_AUTOTUNE chose) and drops the plan's
 * captured graphs, which are captured again by the next call.  The first four
 * do not change the results: every transform runs the same radix passes in the
 * same order, every sweep the same rotations on the same values and both
 * packings the same scalings and roundings; only the split of the work over
 * the threads (or the number of trips through memory) differs.  The ring form
 * computes the same DFTs with other roundings.  HPX_ERR_ARG for other values
 * or an uneven-batch plan. */
int hpx_plan_set_tuning(hpx_plan_s* plan, int ring_elems, int fft_elems, int sweep_form, int pack_pass,
                        int ring_form);

/* Stage timing for profiling.  With profiling enabled (enable = 1) every
 * hpx_analyze records CUDA events on the plan's stream around each of its
 * kernels (ring FFT, poles, NUFFT spreading, NUFFT grid FFT, then either the
 * per-order operators and an empty stage, or with HPX_FLAG_SWEEPS the latitude
 * operator D and the rotation sweeps; up to 256 calls are kept), and every
 * hpx_sh_synthesis around its three stages (the order-m to latitude-Fourier
 * conversion, the type-2 NUFFT, the ring folding and inverse FFTs; the other
 * three stages empty).  hpx_stage_times waits for those events, writes
 * the summed device time of each stage in milliseconds to ms[0..n-1]
 * (n >= HPX_NSTAGES), sets *ncalls to the number of calls summed, and clears
 * the record. */
#define HPX_NSTAGES 6
int hpx_set_profiling(hpx_plan_s* plan, int enable);
int hpx_stage_times(hpx_plan_s* plan, float* ms, int n, int* ncalls);

/* Allocation-free analysis of ONE real FP32 map (the paper has no counterpart;
 * this is a service for callers, not a step of the method).
 *
 * For callers that cannot call cudaMalloc: code running while someone else is
 * capturing the stream into a CUDA graph, plugins whose device memory belongs to
 * a host application's pool, real-time or embedded code that must not allocate
 * after start-up.  It computes the same coefficients as a one-map FP32
 * hpx_analyze plan, but every table and every intermediate buffer lives in one
 * fixed device array inside the library (8 MiB, reserved on every GPU that loads
 * the library until the process exits), so it needs no plan and allocates no
 * device memory.  The caller still passes the input and output buffers:
 *   maps : device float[12 nside^2] (RING order), alm : device float[n_alm][2].
 * Limits: 2 <= nside <= HPX_NOALLOC_MAX_NSIDE (power of two), -1 <= lmax <= 2 nside
 * (-1 = 2 nside); larger sizes return HPX_ERR_NSIDE / HPX_ERR_LMAX.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call before
 * any stream capture.  A call whose nside/lmax differ from the previous call's on
 * the same device rebuilds the tables on the host and copies them into the array
 * (synchronising `cuda_stream`); such a call made while `cuda_stream` is being
 * captured returns HPX_ERR_STATE and touches neither the stream nor the array
 * (make one call of that size before the capture starts).  All calls share the array and it keeps the
 * last call's contents, so calls that overlap on the GPU (different streams or
 * threads) race; serialise them.  Asynchronous on `cuda_stream` otherwise. */
#define HPX_NOALLOC_MAX_NSIDE 128
int hpx_analyze_noalloc(int nside, int lmax, const float* maps, float* alm, void* cuda_stream);

/* Self-test of the failure path (the paper has no counterpart).  Launches one
 * kernel on the plan's stream whose bounded wait on an mbarrier that nothing
 * completes gives up after `spins` polls (1 <= spins <= 2^20) and records
 * HPX_ERR_TIMEOUT in the plan's device status word, exactly as a timed-out
 * wait of the tensor-core kernel does; the next hpx_sync returns
 * HPX_ERR_TIMEOUT and clears the word.  Nothing faults and the context stays
 * usable.  Returns HPX_ERR_ARG for a NULL plan or spins out of range. */
int hpx_selftest_timeout(hpx_plan_s* plan, int spins);

/* Last error code of the calling thread and its message. */
int hpx_last_error(void);
const char* hpx_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* HPX_H */
