// Allocation-free analysis entry point.
//
// Some callers cannot call cudaMalloc at all: code that runs while a CUDA
// stream is being captured into a graph by someone else, plugins hosted inside a
// process whose device memory is owned by a pool or arena they may not touch,
// and real-time or embedded callers that must not allocate after start-up.  For
// them hpx_analyze_noalloc runs the whole analysis of ONE small FP32 map
// (nside <= HPX_NOALLOC_MAX_NSIDE) with every table and every workspace buffer
// carved out of one file-scope device array, g_noalloc_scratch, which the
// library reserves once and every GPU that loads the library keeps until the
// process exits.
//
// In host code the name g_noalloc_scratch is only a host-side stand-in for the
// device array, not a device address; handing it to a kernel would fault (or,
// where the GPU can reach host memory, silently use the wrong memory).  The
// device address is therefore looked up with cudaGetSymbolAddress once per
// device, with that device current, on the first call made on it; that first
// call should come before any stream capture.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/hpx.h"
#include "plan.h"
#include "plan_math.h"

namespace {

constexpr size_t kScratchBytes = (size_t)8 << 20;   // 8 MiB: tables + workspace of one nside-128 map
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Offsets {
    size_t nphi, startN, startS, pow2, logn, fftL, logL, shOff, chOff, bhOff, shift, chirp, bhat, twid,
        poleN, poleS, polew, rowptr, ent, entw, dec, D, angOff, ang, skOff, skew, nstart, swts, shifted;
    size_t Y, bvec;
    int npole;
};

struct DevState {
    unsigned char* base = nullptr;   // device address of g_noalloc_scratch
    int nside = -1, lmax = -1;       // size whose tables the array currently holds
    int nq = 0;
    int spreadE = 0;
    Offsets off;
    hpx::Geometry geo;
};
DevState g_state[kMaxDevices];
std::mutex g_mutex;

// Host image of the tables, laid out as they will sit in the device array.
struct Image {
    std::vector<unsigned char> bytes;
    template <class U>
    size_t put(const U* src, size_t count) {
        const size_t off = align256(bytes.size());
        bytes.resize(off + count * sizeof(U));
        if (count) std::memcpy(bytes.data() + off, src, count * sizeof(U));
        return off;
    }
    template <class U>
    size_t vec(const std::vector<U>& v) { return put(v.data(), v.size()); }
    size_t real(const std::vector<double>& v) {
        std::vector<float> f(v.size());
        for (size_t k = 0; k < v.size(); ++k) f[k] = (float)v[k];
        return vec(f);
    }
};

}  // namespace

// Defined in capi.cu: records the calling thread's last error code.
int hpx_internal_set_error(int code);

namespace {
int fail(int code) { return hpx_internal_set_error(code); }
}  // namespace

extern "C" int hpx_analyze_noalloc(int nside, int lmax, const float* maps, float* alm, void* stream) {
    if (!maps || !alm) return fail(HPX_ERR_ARG);
    if (nside < 2 || nside > HPX_NOALLOC_MAX_NSIDE || (nside & (nside - 1)) != 0) return fail(HPX_ERR_NSIDE);
    const int L = lmax < 0 ? 2 * nside : lmax;
    if (lmax < -1 || L > 2 * nside) return fail(HPX_ERR_LMAX);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fail(HPX_ERR_CUDA);
    std::lock_guard<std::mutex> lock(g_mutex);
    DevState& st = g_state[dev];
    if (!st.base) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return fail(HPX_ERR_CUDA);
        st.base = static_cast<unsigned char*>(p);
    }
    cudaStream_t s = (cudaStream_t)stream;

    if (st.nside != nside || st.lmax != L) {
        // A rebuild copies on the stream and waits for it: not possible while the
        // stream is being captured (the copy would invalidate the caller's capture).
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return fail(HPX_ERR_CUDA);
        if (cs != cudaStreamCaptureStatusNone) return fail(HPX_ERR_STATE);
        // Tables for this size: FP64 on the host, rounded to FP32, packed in the
        // order they take in the device array, followed by the workspace.
        hpx::PlanTables tb;
        Image img;
        Offsets o;
        try {
            if (!hpx::build_tables(nside, L, false, tb).empty()) return fail(HPX_ERR_ARG);
            o.nphi = img.vec(tb.nphi); o.startN = img.vec(tb.startN); o.startS = img.vec(tb.startS);
            o.pow2 = img.vec(tb.pow2); o.logn = img.vec(tb.logn); o.fftL = img.vec(tb.fftL); o.logL = img.vec(tb.logL);
            o.shOff = img.vec(tb.shOff); o.chOff = img.vec(tb.chOff); o.bhOff = img.vec(tb.bhOff);
            o.shift = img.real(tb.shift); o.chirp = img.real(tb.chirp); o.bhat = img.real(tb.bhat);
            o.twid = img.real(tb.twid);
            o.poleN = img.vec(tb.poleN); o.poleS = img.vec(tb.poleS); o.polew = img.vec(tb.polew);
            o.npole = (int)tb.polew.size();
            o.rowptr = img.vec(tb.rowptr); o.ent = img.vec(tb.ent); o.entw = img.real(tb.entw);
            o.dec = img.real(tb.dec); o.D = img.real(tb.D); o.angOff = img.vec(tb.angOff); o.ang = img.real(tb.ang);
            o.skOff = img.vec(tb.skOff); o.skew = img.real(tb.skew); st.nq = tb.nq;
            o.nstart = img.vec(tb.nstart); o.swts = img.real(tb.swts); st.spreadE = tb.spreadE;
            o.shifted = img.vec(tb.shifted);
        } catch (const std::bad_alloc&) {   // no exception leaves the C interface
            return fail(HPX_ERR_OOM);
        } catch (...) {
            return fail(HPX_ERR_ARG);
        }
        const size_t ySize = (size_t)tb.Q * (tb.p + 1) * 8;    // step-1 coefficients (complex FP32)
        const size_t bSize = (size_t)(tb.p + 1) * 2 * tb.P2 * 8;
        o.Y = align256(img.bytes.size());
        o.bvec = o.Y + align256(std::max(ySize, bSize));
        if (o.bvec + align256(bSize) > kScratchBytes) return fail(HPX_ERR_NSIDE);
        st.nside = -1;   // the array is being overwritten
        if (cudaMemcpyAsync(st.base, img.bytes.data(), img.bytes.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(HPX_ERR_CUDA);
        if (cudaStreamSynchronize(s) != cudaSuccess) return fail(HPX_ERR_CUDA);
        hpx::Geometry& g = st.geo;
        g.ns = nside; g.p = tb.p; g.L = L; g.Q = tb.Q; g.npairs = tb.npairs; g.M = tb.M; g.P2 = tb.P2;
        g.Lmax = tb.Lmax; g.smem_ring = tb.smem_ring; g.B = 1; g.npix = tb.npix;
        g.nalm = (int64_t)(L + 1) * (L + 2) / 2;
        st.off = o;
        st.nside = nside;
        st.lmax = L;
    }
    const Offsets& o = st.off;

    // A plan object on the stack whose pointers all lead into the array.
    hpx_plan_s P;
    unsigned char* b = st.base;
    auto& t = P.t;
    t.nphi = (int*)(b + o.nphi); t.startN = (int*)(b + o.startN); t.startS = (int*)(b + o.startS);
    t.pow2 = (int*)(b + o.pow2); t.logn = (int*)(b + o.logn); t.fftL = (int*)(b + o.fftL);
    t.logL = (int*)(b + o.logL); t.shOff = (int64_t*)(b + o.shOff); t.chOff = (int64_t*)(b + o.chOff);
    t.bhOff = (int64_t*)(b + o.bhOff); t.shift = b + o.shift; t.chirp = b + o.chirp; t.bhat = b + o.bhat;
    t.twid = b + o.twid; t.poleN = (int*)(b + o.poleN); t.poleS = (int*)(b + o.poleS);
    t.polew = (double*)(b + o.polew); t.npole = o.npole; t.rowptr = (int*)(b + o.rowptr);
    t.ent = (int*)(b + o.ent); t.entw = b + o.entw; t.dec = b + o.dec; t.D = b + o.D;
    t.angOff = (int64_t*)(b + o.angOff); t.ang = b + o.ang;
    t.skOff = (int64_t*)(b + o.skOff); t.skew = b + o.skew; t.nq = st.nq;
    t.nstart = (int*)(b + o.nstart); t.swts = b + o.swts; t.spreadE = st.spreadE;
    t.shifted = (int*)(b + o.shifted);
    P.g = st.geo;
    P.precision = HPX_FP32;
    P.device = dev;
    P.stream = s;
    P.Y = b + o.Y;
    P.bvec = b + o.bvec;
    P.beta = P.Y;

    hpx::launch_ring_fft<float>(&P, maps, s);
    hpx::launch_poles<float>(&P, maps, s);
    hpx::launch_nufft<float>(&P, s);
    hpx::launch_dense<float>(&P, s);
    hpx::launch_rot<float>(&P, alm, s);
    if (cudaGetLastError() != cudaSuccess) return fail(HPX_ERR_CUDA);
    return fail(HPX_OK);
}
