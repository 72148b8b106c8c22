// C ABI of the HP2SPH library (include/hpx.h): plan construction, table upload,
// and the launch sequences of Algorithm 1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/hpx.h"
#include "plan.h"
#include "plan_math.h"

namespace {

thread_local int g_last_error = HPX_OK;

// ring transforms of at most this many points run in one launch (blocks of
// kRingMergeN / 16 threads)
constexpr int kRingMergeN = 2048;

int set_err(int code) {
    g_last_error = code;
    return code;
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

struct Uploader {
    hpx_plan_s* P;
    bool ok = true;
    template <class U>
    U* raw(const U* src, size_t count) {
        if (!ok || count == 0) return nullptr;
        U* d = nullptr;
        if (cudaMalloc(&d, count * sizeof(U)) != cudaSuccess) { ok = false; return nullptr; }
        P->bytes += (int64_t)(count * sizeof(U));
        if (cudaMemcpy(d, src, count * sizeof(U), cudaMemcpyHostToDevice) != cudaSuccess) { ok = false; }
        return d;
    }
    template <class U>
    U* vec(const std::vector<U>& v) { return raw(v.data(), v.size()); }
    // double table -> device table of the plan precision
    void* real(const std::vector<double>& v, bool fp64) {
        if (fp64) return vec(v);
        std::vector<float> f(v.size());
        for (size_t k = 0; k < v.size(); ++k) f[k] = (float)v[k];
        return vec(f);
    }
};

void free_plan(hpx_plan_s* P) {
    if (!P) return;
    for (auto& e : P->graphs) cudaGraphExecDestroy(e.exec);
    if (P->group) {
        // after a graph capture the sub-plans still name the group's capture
        // stream: finish it and let them synchronise on the legacy stream
        if (P->cap) cudaStreamSynchronize(P->cap);
        for (hpx_plan_s* S : P->subs) S->stream = nullptr;
        hpx::group_free(P);
        if (P->d_status) cudaFree(P->d_status);
        if (P->cap) cudaStreamDestroy(P->cap);
        delete P;
        return;
    }
    if (P->cap) cudaStreamDestroy(P->cap);
    auto& t = P->t;
    void* ptrs[] = {t.nphi, t.startN, t.startS, t.pow2, t.logn, t.fftL, t.logL, t.shOff, t.chOff,
                    t.bhOff, t.shift, t.chirp, t.bhat, t.twid, t.ch4Off, t.bh4Off, t.chirp4, t.bhat4, t.poleN,
                    t.poleS, t.polew, t.rowptr,
                    t.ent, t.entw, t.dec, t.D, t.tstart, t.hwn, t.angOff, t.ang, t.skOff, t.skew, t.skewT, t.nrowptr, t.nent, t.nentw, t.nstart, t.swts, t.hstart, t.hwts, t.Es, t.shifted, t.C, t.cgH, P->Y, P->U, P->bvec,
                    P->fusedM, P->fusedOff, P->fusedTiles, P->tcOff, P->tcFirst, P->tcRinv, P->bscale, P->d_status, P->synM, P->ringList,
                    P->jres, P->jalm, P->dTC, P->dRinv, P->dTiles, P->dTcOff, P->mapIdx, P->bpk, P->synT,
                    P->synRinv, P->synTiles, P->synNch, P->synOff, P->synRowBase, P->synScale, P->synBpk};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (P->ev) {
        for (int k = 0; k < hpx_plan_s::kMaxProf * (hpx_plan_s::kStages + 1); ++k) cudaEventDestroy(P->ev[k]);
        delete[] P->ev;
    }
    delete P;
}

template <class T>
int analyze_impl(hpx_plan_s* P, const void* maps, void* alm, bool rings = true) {
    cudaStream_t s = P->stream;
    cudaEvent_t* ev = nullptr;
    if (P->prof && P->nprof < hpx_plan_s::kMaxProf) ev = P->ev + (size_t)P->nprof++ * (hpx_plan_s::kStages + 1);
    if (ev) cudaEventRecord(ev[0], s);
    if (rings) hpx::launch_ring_fft<T>(P, (const T*)maps, s);
    if (ev) cudaEventRecord(ev[1], s);
    hpx::launch_poles<T>(P, (const T*)maps, s);
    if (ev) cudaEventRecord(ev[2], s);
    hpx::launch_spread<T>(P, s);
    if (ev) cudaEventRecord(ev[3], s);
    hpx::launch_lat_fft<T>(P, s, hpx::packs_b(P));
    if (ev) cudaEventRecord(ev[4], s);
    if (P->fusedM) {
        if constexpr (sizeof(T) == 4) {
            if (P->use_tc) hpx::launch_fused_tc(P, (float*)alm, s);
            else hpx::launch_fused<T>(P, (T*)alm, s);
        } else {
            hpx::launch_fused<T>(P, (T*)alm, s);
        }
        if (ev) cudaEventRecord(ev[5], s);
    } else {
        if (P->flags & HPX_FLAG_CG) {
            hpx::launch_cg<T>(P, s);                  // bvec <- T^{-1} bvec, column by column
            hpx::launch_dense<T>(P, s, P->t.C);       // change of basis alone
        } else if (sizeof(T) == 4 && P->dTC) {
            hpx::launch_dense_tc(P, s);               // D on the tensor cores
        } else {
            hpx::launch_dense<T>(P, s);
        }
        if (ev) cudaEventRecord(ev[5], s);
        hpx::launch_rot<T>(P, (T*)alm, s);
    }
    if (ev) cudaEventRecord(ev[6], s);
    if (cudaGetLastError() != cudaSuccess) return HPX_ERR_CUDA;
    return HPX_OK;
}

}  // namespace

int hpx_internal_set_error(int code) { return set_err(code); }

namespace hpx {
int analyze_after_rings(hpx_plan_s* P, const void* maps, void* alm) {
    return P->precision == HPX_FP64 ? analyze_impl<double>(P, maps, alm, false)
                                    : analyze_impl<float>(P, maps, alm, false);
}
}  // namespace hpx

namespace {
int autotune(hpx_plan_s* P);
}  // namespace

extern "C" {

hpx_plan_s* hpx_plan_ex(const hpx_plan_desc* d) {
    if (!d) { set_err(HPX_ERR_ARG); return nullptr; }
    if ((d->flags & ~(unsigned)(HPX_FLAG_SWEEPS | HPX_FLAG_GRAPH | HPX_FLAG_SIMT | HPX_FLAG_CHECKED |
                                HPX_FLAG_AUTOTUNE | HPX_FLAG_SYNTHESIS | HPX_FLAG_CG | HPX_FLAG_JACOBI)) != 0 ||
        d->batch < 1) {
        set_err(HPX_ERR_ARG);
        return nullptr;
    }
    if (d->flags & HPX_FLAG_JACOBI) {   // the Jacobi iteration needs the synthesis
        hpx_plan_desc dj = *d;
        dj.flags = (d->flags & ~HPX_FLAG_JACOBI) | HPX_FLAG_SYNTHESIS;
        if (d->nsides || d->lmaxs) { set_err(HPX_ERR_ARG); return nullptr; }   // uniform plans only
        hpx_plan_s* P = hpx_plan_ex(&dj);
        if (!P) return nullptr;
        const size_t es = d->precision == HPX_FP64 ? 8 : 4;
        if (cudaMalloc(&P->jres, (size_t)P->g.B * P->g.npix * es) != cudaSuccess ||
            cudaMalloc(&P->jalm, (size_t)P->g.B * P->g.nalm * 2 * es) != cudaSuccess) {
            cudaGetLastError();
            free_plan(P);
            set_err(HPX_ERR_OOM);
            return nullptr;
        }
        P->bytes += (int64_t)((size_t)P->g.B * P->g.npix * es + (size_t)P->g.B * P->g.nalm * 2 * es);
        P->flags |= HPX_FLAG_JACOBI;
        set_err(HPX_OK);
        return P;
    }
    if (d->precision != HPX_FP32 && d->precision != HPX_FP64) { set_err(HPX_ERR_ARG); return nullptr; }
    if (d->nsides || d->lmaxs) {
        int err = HPX_OK;
        hpx_plan_s* G = hpx::group_create(d, &err);
        if (!G) { set_err(err); return nullptr; }
        if (!hpx::group_build_ring_list(G)) {
            cudaGetLastError();
            free_plan(G);
            set_err(HPX_ERR_OOM);
            return nullptr;
        }
        if (cudaMalloc(&G->d_status, sizeof(int)) != cudaSuccess) {
            free_plan(G);
            set_err(HPX_ERR_OOM);
            return nullptr;
        }
        cudaMemset(G->d_status, 0, sizeof(int));
        if ((d->flags & HPX_FLAG_GRAPH) && cudaStreamCreateWithFlags(&G->cap, cudaStreamNonBlocking) != cudaSuccess) {
            free_plan(G);
            set_err(HPX_ERR_CUDA);
            return nullptr;
        }
        set_err(HPX_OK);
        return G;
    }
    const int ns = d->nside;
    const bool fp64 = d->precision == HPX_FP64;
    if (d->precision != HPX_FP32 && d->precision != HPX_FP64) { set_err(HPX_ERR_ARG); return nullptr; }
    if (!is_pow2(ns) || ns < 2 || ns > (fp64 ? 1024 : 2048)) { set_err(HPX_ERR_NSIDE); return nullptr; }
    const int L = d->lmax < 0 ? 2 * ns : d->lmax;
    if (L > 2 * ns) { set_err(HPX_ERR_LMAX); return nullptr; }
    if (d->lmax < -1) { set_err(HPX_ERR_LMAX); return nullptr; }

    hpx::PlanTables tb;
    std::string msg;
    try {
        msg = hpx::build_tables(ns, L, fp64, tb);
    } catch (const std::bad_alloc&) {
        set_err(HPX_ERR_OOM);
        return nullptr;
    } catch (...) {
        set_err(HPX_ERR_ARG);
        return nullptr;
    }
    if (!msg.empty()) { set_err(HPX_ERR_ARG); return nullptr; }

    hpx_plan_s* P = new (std::nothrow) hpx_plan_s();
    if (!P) { set_err(HPX_ERR_OOM); return nullptr; }
    P->precision = d->precision;
    cudaGetDevice(&P->device);
    P->stream = nullptr;
    auto& g = P->g;
    g.ns = ns; g.p = tb.p; g.L = L; g.Q = tb.Q; g.npairs = tb.npairs; g.M = tb.M; g.P2 = tb.P2;
    g.Lmax = tb.Lmax; g.smem_ring = tb.smem_ring; g.B = d->batch; g.npix = tb.npix;
    g.nalm = (int64_t)(L + 1) * (L + 2) / 2;

    Uploader up{P};
    auto& t = P->t;
    t.nphi = up.vec(tb.nphi); t.startN = up.vec(tb.startN); t.startS = up.vec(tb.startS);
    t.pow2 = up.vec(tb.pow2); t.logn = up.vec(tb.logn); t.fftL = up.vec(tb.fftL); t.logL = up.vec(tb.logL);
    t.shOff = up.vec(tb.shOff); t.chOff = up.vec(tb.chOff); t.bhOff = up.vec(tb.bhOff);
    t.shift = up.real(tb.shift, fp64); t.chirp = up.real(tb.chirp, fp64); t.bhat = up.real(tb.bhat, fp64);
    t.ch4Off = up.vec(tb.ch4Off); t.bh4Off = up.vec(tb.bh4Off);
    t.chirp4 = up.real(tb.chirp4, fp64); t.bhat4 = up.real(tb.bhat4, fp64);
    t.twid = up.real(tb.twid, fp64);
    t.poleN = up.vec(tb.poleN); t.poleS = up.vec(tb.poleS); t.polew = up.vec(tb.polew);
    t.npole = (int)tb.polew.size();
    {   // ring pairs grouped by transform length (longest first), and from
        // kRingCtMin points up also by kind (plain rings, then Bluestein rings)
        struct Key {
            int N, blue, i;
        };
        std::vector<Key> byN;
        for (int i = 0; i < tb.npairs; ++i)
            byN.push_back({tb.pow2[i] ? tb.nphi[i] : tb.fftL[i], tb.pow2[i] ? 0 : 1, i});
        std::stable_sort(byN.begin(), byN.end(), [](const Key& a, const Key& b) {
            if (a.N != b.N) return a.N > b.N;
            return a.N >= hpx::kRingCtMin && a.blue < b.blue;
        });
        std::vector<int> list;
        for (size_t k = 0; k < byN.size(); ++k) {
            // transforms of kRingMergeN points or fewer share one launch, with
            // blocks sized for the longest of them: alone, each of these short
            // launches is bound by its latency, not by its work
            const bool merged = byN[k].N <= kRingMergeN && k > 0 && byN[k - 1].N <= kRingMergeN;
            const bool newkind = byN[k].N >= hpx::kRingCtMin && k > 0 && byN[k].blue != byN[k - 1].blue;
            if (k == 0 || (byN[k].N != byN[k - 1].N && !merged) || newkind)
                P->ringClasses.push_back({byN[k].N, (int)k, 0, byN[k].blue != 0});
            P->ringClasses.back().count++;
            list.push_back(byN[k].i);
        }
        P->ringList = up.vec(list);
    }
    t.rowptr = up.vec(tb.rowptr); t.ent = up.vec(tb.ent);
    t.entw = up.real(tb.entw, fp64); t.dec = up.real(tb.dec, fp64);
    t.nstart = up.vec(tb.nstart); t.swts = up.real(tb.swts, fp64); t.spreadE = tb.spreadE;
    t.hstart = up.vec(tb.hstart); t.hwts = up.real(tb.hwts, fp64); t.spreadH = tb.spreadH;
    t.tstart = up.vec(tb.tstart); t.hwn = up.real(tb.hwn, fp64); t.interpE = tb.interpE;
    t.interpRows = tb.interpRows;
    t.interpD = tb.interpD;
    t.spreadRows = tb.spreadRows;
    t.spreadD = tb.spreadD;
    t.D = up.real(tb.D, fp64);
    if (d->flags & HPX_FLAG_CG) {
        std::vector<double> H;
        hpx::build_cg_tables(tb, t.cgN, H, t.cgk0, t.cgn);
        t.cgH = up.real(H, fp64);
        t.C = up.real(tb.C, fp64);
    }
    t.shifted = up.vec(tb.shifted);
    std::vector<double> EsHost;
    if (d->flags & HPX_FLAG_SYNTHESIS) {
        hpx::build_synthesis_table(tb, EsHost);
        t.Es = up.real(EsHost, fp64);
    }
    t.angOff = up.vec(tb.angOff); t.ang = up.real(tb.ang, fp64);
    t.skOff = up.vec(tb.skOff); t.skew = up.real(tb.skew, fp64); t.nq = tb.nq;
    t.skewT = up.real(tb.skewT, fp64);
    t.nrowptr = up.vec(tb.nrowptr); t.nent = up.vec(tb.nent); t.nentw = up.real(tb.nentw, fp64);
    if (!up.ok) { free_plan(P); set_err(HPX_ERR_OOM); return nullptr; }

    const size_t es = fp64 ? 16 : 8;   // complex element
    const size_t ySize = (size_t)g.B * g.Q * (g.p + 1) * es;
    const size_t bSize = (size_t)g.B * (g.p + 1) * 2 * g.P2 * es;
    if (cudaMalloc(&P->Y, std::max(ySize, bSize)) != cudaSuccess) { free_plan(P); set_err(HPX_ERR_OOM); return nullptr; }
    if (cudaMalloc(&P->bvec, bSize) != cudaSuccess) { free_plan(P); set_err(HPX_ERR_OOM); return nullptr; }
    P->beta = P->Y;   // Y is dead once the NUFFT has read it
    P->ldu = (g.M / 2 + 2) & ~1;
    const size_t uSize = (size_t)g.B * (g.L + 1) * P->ldu * es;
    if (cudaMalloc(&P->U, uSize) != cudaSuccess) { free_plan(P); set_err(HPX_ERR_OOM); return nullptr; }
    P->bytes += (int64_t)(std::max(ySize, bSize) + bSize + uSize);
    P->flags = d->flags;
    if (cudaMalloc(&P->d_status, sizeof(int)) != cudaSuccess) { free_plan(P); set_err(HPX_ERR_OOM); return nullptr; }
    cudaMemset(P->d_status, 0, sizeof(int));
    if ((d->flags & HPX_FLAG_GRAPH) && cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking) != cudaSuccess) {
        free_plan(P);
        set_err(HPX_ERR_CUDA);
        return nullptr;
    }
    if (d->flags & HPX_FLAG_CG) P->flags |= HPX_FLAG_SWEEPS;   // CG runs with the per-call sweeps
    if (!(P->flags & HPX_FLAG_SWEEPS)) {
        // per-order operators; without room for them the plan keeps the sweeps
        std::vector<int64_t> off((size_t)(L + 1) * 2 + 1, 0);
        std::vector<int> tiles;
        const int rows = hpx::fused_tile_rows(g.B);
        for (int m = 0; m <= L; ++m)
            for (int c = 0; c < 2; ++c) {
                const int n = hpx::chain_len(m, c, L);
                off[(size_t)m * 2 + c + 1] = off[(size_t)m * 2 + c] + n;
                for (int i0 = 0; i0 < n; i0 += rows) { tiles.push_back(m); tiles.push_back(c); tiles.push_back(i0); }
            }
        P->fused_ldm = (g.P2 + 3) / 4 * 4;
        size_t mBytes = (size_t)off.back() * P->fused_ldm * (fp64 ? 8 : 4);
        P->use_tc = !fp64 && g.B > 8 && !(d->flags & HPX_FLAG_SIMT);
        std::vector<int64_t> tcOff;
        std::vector<int> tcFirst;
        if (P->use_tc) {   // tiles of 128 rows, K-chunks of 32 in the MMA's layout
            const int64_t nch = (g.P2 + 31) / 32;
            int64_t o = 0;
            tcFirst.assign((size_t)(L + 1) * 2, 0);
            for (size_t q = 0; q < tiles.size(); q += 3) {
                const int m = tiles[q], c = tiles[q + 1], i0 = tiles[q + 2];
                if (i0 == 0) tcFirst[(size_t)m * 2 + c] = (int)(q / 3);
                const int rows = std::min(128, hpx::chain_len(m, c, L) - i0);
                tcOff.push_back(o);
                o += nch * ((rows + 7) & ~7) * 32;
            }
            mBytes = (size_t)o * 4;
        }
        size_t freeB = 0, totalB = 0;
        cudaMemGetInfo(&freeB, &totalB);
        // operators above 24 GB (nside 2048: 69 GB, ~4 minutes of FP64 build) are
        // not built by default: the per-call sweeps are used instead
        const bool fits = mBytes <= ((size_t)24 << 30) && mBytes + ((size_t)1 << 30) < freeB;
        if (fits && cudaMalloc(&P->fusedM, mBytes) == cudaSuccess) {
            P->bytes += (int64_t)mBytes;
            P->fused_bytes = (int64_t)mBytes;
            cudaMemset(P->fusedM, 0, mBytes);   // zero the row padding
            P->fusedOff = up.vec(off);
            P->fusedTiles = up.vec(tiles);
            P->fused_ntiles = (int)(tiles.size() / 3);
            if (P->use_tc) {
                P->tcOff = up.vec(tcOff);
                P->tcFirst = up.vec(tcFirst);
            }
            double* D64 = (double*)t.D;
            hpx::cplx<double>* sk64 = (hpx::cplx<double>*)t.skew;
            if (!fp64) { D64 = up.vec(tb.D); sk64 = (hpx::cplx<double>*)up.vec(tb.skew); }
            int rc = up.ok ? (fp64 ? hpx::build_fused<double>(P, D64, sk64, nullptr, P->fusedM, P->use_tc)
                                   : hpx::build_fused<float>(P, D64, sk64, nullptr, P->fusedM, P->use_tc))
                           : -1;
            if (rc == 0 && P->use_tc) rc = hpx::prepare_fused_tc(P);
            // synthesis operators R_{m,c} Es (row-major), when asked for and room allows
            const size_t sBytes = (size_t)off.back() * P->fused_ldm * (fp64 ? 8 : 4);
            cudaMemGetInfo(&freeB, &totalB);
            if (rc == 0 && (d->flags & HPX_FLAG_SYNTHESIS) && sBytes + ((size_t)1 << 30) < freeB &&
                cudaMalloc(&P->synM, sBytes) == cudaSuccess) {
                P->bytes += (int64_t)sBytes;
                cudaMemset(P->synM, 0, sBytes);
                double* Es64 = fp64 ? (double*)t.Es : up.vec(EsHost);
                rc = up.ok ? (fp64 ? hpx::build_fused<double>(P, Es64, sk64, nullptr, P->synM, false)
                                   : hpx::build_fused<float>(P, Es64, sk64, nullptr, P->synM, false))
                           : -1;
                if (!fp64 && Es64) { cudaFree(Es64); P->bytes -= (int64_t)(EsHost.size() * 8); }
                // FP32 plans on the tensor cores apply them there too
                if (rc == 0 && P->use_tc) rc = hpx::prepare_synth_tc(P);
            } else {
                cudaGetLastError();
            }
            if (!fp64) {
                if (D64) { cudaFree(D64); P->bytes -= (int64_t)(tb.D.size() * 8); }
                if (sk64) { cudaFree(sk64); P->bytes -= (int64_t)(tb.skew.size() * 8); }
            }
            if (rc != 0 || !up.ok) { free_plan(P); set_err(HPX_ERR_CUDA); return nullptr; }
        } else {
            P->fusedM = nullptr;
            cudaGetLastError();
            P->flags |= HPX_FLAG_SWEEPS;
        }
    }
    if (cudaDeviceSynchronize() != cudaSuccess) { free_plan(P); set_err(HPX_ERR_CUDA); return nullptr; }
    if (d->flags & HPX_FLAG_AUTOTUNE) {
        const int rc = autotune(P);
        if (rc != HPX_OK) { free_plan(P); set_err(rc); return nullptr; }
    }
    // the sweeps path of FP32 plans of 4 maps or more: D on the tensor cores (its
    // tiles are 32 maps wide; below 4 maps the FP32-pipe kernel is as fast).  Up
    // to nside 1024: at nside 2048 (K = 2049 terms per row) the FP16 pairs' 2^-22
    // representation error of both operands left a flat-spectrum map at 1.2e-5
    // per degree, above the 1e-5 of FP32 plans, so the FP32 pipes apply D there
    if (!P->fusedM && !fp64 && g.B >= 4 && ns <= 1024 && !(d->flags & (HPX_FLAG_SIMT | HPX_FLAG_CG)) &&
        hpx::prepare_dense_tc(P) != 0) {
        free_plan(P);
        set_err(HPX_ERR_CUDA);
        return nullptr;
    }
    set_err(HPX_OK);
    return P;
}

hpx_plan_s* hpx_plan(int nside, int lmax, int batch) {
    hpx_plan_desc d;
    std::memset(&d, 0, sizeof(d));
    d.nside = nside;
    d.lmax = lmax;
    d.batch = batch;
    d.precision = HPX_FP32;
    return hpx_plan_ex(&d);
}

int hpx_set_stream(hpx_plan_s* P, void* stream) {
    if (!P) return set_err(HPX_ERR_ARG);
    P->stream = (cudaStream_t)stream;
    return set_err(HPX_OK);
}

}  // extern "C"

namespace {

int analyze_direct(hpx_plan_s* P, const void* maps, void* alm) {
    if (P->flags & HPX_FLAG_CHECKED) {
        const int64_t n = P->group ? P->total_npix : P->g.npix * P->g.B;
        hpx::launch_finite_check(maps, n, P->precision == HPX_FP64, P->d_status, P->stream);
    }
    if (P->group) return hpx::group_analyze(P, maps, alm);
    return P->precision == HPX_FP64 ? analyze_impl<double>(P, maps, alm) : analyze_impl<float>(P, maps, alm);
}

// Launch shapes chosen by HPX_FLAG_AUTOTUNE, per (nside, lmax, batch,
// precision): later plans of the same shape reuse them without timing.
struct TuneKey {
    int ns, L, B, prec;
    bool operator<(const TuneKey& o) const {
        return std::tie(ns, L, B, prec) < std::tie(o.ns, o.L, o.B, o.prec);
    }
};
struct TuneVal {
    int ringE, latE, rotForm, packSep, ringForm;   // shapes, sweep form, b packing, Bluestein ring form
};
std::mutex g_tune_mutex;
std::map<TuneKey, TuneVal> g_tune_cache;

// Times one stage (ring FFT: stage 0, grid FFT: stage 1, run-time sweeps:
// stage 2, writing into the scratch alm) of the analysis with the plan's
// current launch shape: one warm-up, then the best of three.
float time_stage(hpx_plan_s* P, const void* maps, void* alm, int stage, cudaEvent_t e0, cudaEvent_t e1) {
    float best = 0.f;
    for (int r = 0; r < 4; ++r) {
        cudaEventRecord(e0, P->stream);
        if (P->precision == HPX_FP64) {
            if (stage == 0) hpx::launch_ring_fft<double>(P, (const double*)maps, P->stream);
            else hpx::launch_lat_fft<double>(P, P->stream);
        } else {
            if (stage == 0) hpx::launch_ring_fft<float>(P, (const float*)maps, P->stream);
            else if (stage == 1) hpx::launch_lat_fft<float>(P, P->stream, hpx::packs_b(P));
            else hpx::launch_rot<float>(P, (float*)alm, P->stream);
        }
        cudaEventRecord(e1, P->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r == 1 || (r > 1 && ms < best)) best = ms;
    }
    return best;
}

void tune_shapes(hpx_plan_s* P, const void* maps, void* alm, cudaEvent_t e0, cudaEvent_t e1) {
    const bool sweeps = !P->fusedM && P->precision == HPX_FP32;   // the FP32 run-time sweeps run per call
    const TuneKey key{P->g.ns, P->g.L, P->g.B, P->precision * 2 + (sweeps ? 1 : 0)};
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            P->ringE = it->second.ringE;
            P->latE = it->second.latE;
            P->rotForm = it->second.rotForm;
            P->packSep = it->second.packSep;
            P->ringForm = it->second.ringForm;
            return;
        }
    }
    float t[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int e = 0; e < 2; ++e) {
        P->ringE = P->latE = e ? 32 : 16;
        t[0][e] = time_stage(P, maps, alm, 0, e0, e1);
        t[1][e] = time_stage(P, maps, alm, 1, e0, e1);
    }
    P->ringE = t[0][1] < t[0][0] ? 32 : 16;
    P->latE = t[1][1] < t[1][0] ? 32 : 16;
    {   // the Bluestein ring classes: whole-ring or quarter-length convolutions
        P->ringForm = 1;
        const float t4 = time_stage(P, maps, alm, 0, e0, e1);
        P->ringForm = t4 < t[0][P->ringE == 32 ? 1 : 0] ? 1 : 0;
    }
    P->rotForm = 0;
    if (sweeps) {   // the three forms of the sweep kernel
        float best = 0.f;
        for (int f = 0; f < 3; ++f) {
            const int keep = P->rotForm;
            P->rotForm = f;
            const float tf = time_stage(P, maps, alm, 2, e0, e1);
            if (f == 0 || tf < best) best = tf;
            else P->rotForm = keep;
        }
    }
    // packed b for the tensor cores: in the grid-FFT kernel or in a pass of its own
    if (hpx::packs_b(P)) {
        P->packSep = 0;
        const float tin = time_stage(P, maps, alm, 1, e0, e1);
        P->packSep = 1;
        const float tsep = time_stage(P, maps, alm, 1, e0, e1);
        P->packSep = tsep < tin ? 1 : 0;
    }
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = {P->ringE, P->latE, P->rotForm, P->packSep, P->ringForm};
}

// HPX_FLAG_AUTOTUNE: choose the launch shapes of the FFT stages (tune_shapes),
// then time the operator path and the run-time sweeps on scratch buffers (3
// analyses each after one warm-up) and keep the faster.
int autotune(hpx_plan_s* P) {
    const size_t es = P->precision == HPX_FP64 ? 8 : 4;
    void *maps = nullptr, *alm = nullptr;
    if (cudaMalloc(&maps, (size_t)P->g.B * P->g.npix * es) != cudaSuccess) return HPX_ERR_OOM;
    if (cudaMalloc(&alm, (size_t)P->g.B * P->g.nalm * es * 2) != cudaSuccess) {
        cudaFree(maps);
        return HPX_ERR_OOM;
    }
    cudaMemset(maps, 0, (size_t)P->g.B * P->g.npix * es);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    tune_shapes(P, maps, alm, e0, e1);
    if (!P->fusedM) {   // only the sweeps: nothing else to choose
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(maps);
        cudaFree(alm);
        return cudaGetLastError() == cudaSuccess ? HPX_OK : HPX_ERR_CUDA;
    }
    float ms[2] = {0.f, 0.f};
    void* M = P->fusedM;
    for (int path = 0; path < 2; ++path) {   // 0: operators, 1: sweeps
        P->fusedM = path == 0 ? M : nullptr;
        analyze_direct(P, maps, alm);
        cudaEventRecord(e0, P->stream);
        for (int r = 0; r < 3; ++r) analyze_direct(P, maps, alm);
        cudaEventRecord(e1, P->stream);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms[path], e0, e1);
    }
    P->fusedM = M;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(maps);
    cudaFree(alm);
    if (cudaGetLastError() != cudaSuccess) return HPX_ERR_CUDA;
    P->tuned_ms[0] = ms[0] / 3;
    P->tuned_ms[1] = ms[1] / 3;
    if (ms[1] < ms[0]) {   // keep the sweeps: release the operators
        void* ptrs[] = {P->fusedM, P->synM ? nullptr : P->fusedOff, P->fusedTiles, P->tcOff, P->tcFirst,
                        P->tcRinv, P->bscale, P->bpk};
        for (void* q : ptrs)
            if (q) cudaFree(q);
        P->fusedM = nullptr;
        if (!P->synM) P->fusedOff = nullptr;
        P->fusedTiles = nullptr;
        P->tcOff = nullptr;
        P->tcFirst = nullptr;
        P->tcRinv = nullptr;
        P->bscale = nullptr;
        P->bpk = nullptr;
        P->bytes -= P->fused_bytes;
        P->fused_bytes = 0;
        P->use_tc = false;
        P->flags |= HPX_FLAG_SWEEPS;
    }
    return HPX_OK;
}

// HPX_FLAG_CHECKED, host side: both pointers must be device (or managed) memory
// of the plan's device.
bool device_pointer(const hpx_plan_s* P, const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == P->device;
}

// HPX_FLAG_GRAPH: replay the graph captured for this (maps, alm) pair, or
// capture the launch sequence on the plan's own stream first.
int analyze_graph(hpx_plan_s* P, const void* maps, void* alm) {
    for (auto& e : P->graphs)
        if (e.maps == maps && e.alm == alm)
            return cudaGraphLaunch(e.exec, P->stream) == cudaSuccess ? HPX_OK : HPX_ERR_CUDA;
    cudaStream_t user = P->stream;
    const bool prof = P->prof;
    P->stream = P->cap;
    P->prof = false;
    if (cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        P->stream = user;
        P->prof = prof;
        return HPX_ERR_CUDA;
    }
    const int rc = analyze_direct(P, maps, alm);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(P->cap, &graph);
    P->stream = user;
    P->prof = prof;
    if (rc != HPX_OK || ec != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        return rc != HPX_OK ? rc : HPX_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return HPX_ERR_CUDA;
    P->graphs.push_back({maps, alm, exec});
    return cudaGraphLaunch(exec, P->stream) == cudaSuccess ? HPX_OK : HPX_ERR_CUDA;
}

}  // namespace

extern "C" {

int hpx_analyze(hpx_plan_s* P, const void* maps, void* alm) {
    if (!P || !maps || !alm) return set_err(HPX_ERR_ARG);
    if ((P->flags & HPX_FLAG_CHECKED) && (!device_pointer(P, maps) || !device_pointer(P, alm)))
        return set_err(HPX_ERR_ARG);
    const int rc = (P->flags & HPX_FLAG_GRAPH) ? analyze_graph(P, maps, alm) : analyze_direct(P, maps, alm);
    return set_err(rc);
}

int hpx_synthesize(hpx_plan_s* P, const void* alm, void* maps) {
    if (!P || !alm || !maps) return set_err(HPX_ERR_ARG);
    if (P->flags & HPX_FLAG_CHECKED) {
        if (!device_pointer(P, maps) || !device_pointer(P, alm)) return set_err(HPX_ERR_ARG);
        const int64_t n = 2 * (P->group ? P->total_nalm : P->g.nalm * P->g.B);
        hpx::launch_finite_check(alm, n, P->precision == HPX_FP64, P->d_status, P->stream);
    }
    if (P->group) return set_err(hpx::group_synthesize(P, alm, maps));
    if (P->precision == HPX_FP64) hpx::launch_adjoint<double>(P, (const double*)alm, (double*)maps, P->stream);
    else hpx::launch_adjoint<float>(P, (const float*)alm, (float*)maps, P->stream);
    if (cudaGetLastError() != cudaSuccess) return set_err(HPX_ERR_CUDA);
    return set_err(HPX_OK);
}

int hpx_analyze_vjp(hpx_plan_s* P, const void* galm, void* gmaps) {
    if (!P || !galm || !gmaps) return set_err(HPX_ERR_ARG);
    if (P->flags & HPX_FLAG_CHECKED) {
        if (!device_pointer(P, gmaps) || !device_pointer(P, galm)) return set_err(HPX_ERR_ARG);
        const int64_t n = 2 * (P->group ? P->total_nalm : P->g.nalm * P->g.B);
        hpx::launch_finite_check(galm, n, P->precision == HPX_FP64, P->d_status, P->stream);
    }
    if (P->group) return set_err(hpx::group_analyze_vjp(P, galm, gmaps));
    if (P->precision == HPX_FP64) hpx::launch_adjoint<double>(P, (const double*)galm, (double*)gmaps, P->stream, 1.0);
    else hpx::launch_adjoint<float>(P, (const float*)galm, (float*)gmaps, P->stream, 1.0f);
    if (cudaGetLastError() != cudaSuccess) return set_err(HPX_ERR_CUDA);
    return set_err(HPX_OK);
}

int hpx_cl_vjp(hpx_plan_s* P, const void* alm, const double* gcl, void* galm) {
    if (!P || !alm || !gcl || !galm) return set_err(HPX_ERR_ARG);
    if ((P->flags & HPX_FLAG_CHECKED) &&
        (!device_pointer(P, alm) || !device_pointer(P, gcl) || !device_pointer(P, galm)))
        return set_err(HPX_ERR_ARG);
    const int64_t* ao = P->group ? P->d_almel : nullptr;
    const int64_t* co = P->group ? P->d_clel : nullptr;
    const int* lm = P->group ? P->d_lmax : nullptr;
    if (P->precision == HPX_FP64)
        hpx::launch_cl_vjp<double>((const double*)alm, gcl, (double*)galm, ao, co, lm, P->g.L, P->g.B, P->g.L,
                                   P->g.nalm, P->stream);
    else
        hpx::launch_cl_vjp<float>((const float*)alm, gcl, (float*)galm, ao, co, lm, P->g.L, P->g.B, P->g.L,
                                  P->g.nalm, P->stream);
    if (cudaGetLastError() != cudaSuccess) return set_err(HPX_ERR_CUDA);
    return set_err(HPX_OK);
}

int hpx_sh_synthesis(hpx_plan_s* P, const void* alm, void* maps) {
    if (!P || !alm || !maps) return set_err(HPX_ERR_ARG);
    if (!(P->flags & HPX_FLAG_SYNTHESIS)) return set_err(HPX_ERR_STATE);
    if (P->flags & HPX_FLAG_CHECKED) {
        if (!device_pointer(P, maps) || !device_pointer(P, alm)) return set_err(HPX_ERR_ARG);
        const int64_t n = 2 * (P->group ? P->total_nalm : P->g.nalm * P->g.B);
        hpx::launch_finite_check(alm, n, P->precision == HPX_FP64, P->d_status, P->stream);
    }
    if (P->group) return set_err(hpx::group_sh_synthesis(P, alm, maps));
    cudaEvent_t* ev = nullptr;
    if (P->prof && P->nprof < hpx_plan_s::kMaxProf) ev = P->ev + (size_t)P->nprof++ * (hpx_plan_s::kStages + 1);
    if (P->precision == HPX_FP64)
        hpx::launch_sh_synthesis<double>(P, (const double*)alm, (double*)maps, P->stream, ev);
    else
        hpx::launch_sh_synthesis<float>(P, (const float*)alm, (float*)maps, P->stream, ev);
    if (cudaGetLastError() != cudaSuccess) return set_err(HPX_ERR_CUDA);
    return set_err(HPX_OK);
}

int hpx_sh_synthesis_adjoint(hpx_plan_s* P, const void* maps, void* alm) {
    if (!P || !alm || !maps) return set_err(HPX_ERR_ARG);
    if (P->group || !(P->flags & HPX_FLAG_SYNTHESIS)) return set_err(HPX_ERR_STATE);
    if ((P->flags & HPX_FLAG_CHECKED) && (!device_pointer(P, maps) || !device_pointer(P, alm)))
        return set_err(HPX_ERR_ARG);
    if (P->precision == HPX_FP64) hpx::launch_sh_adjoint<double>(P, (const double*)maps, (double*)alm, P->stream, 1.0);
    else hpx::launch_sh_adjoint<float>(P, (const float*)maps, (float*)alm, P->stream, 1.0f);
    if (cudaGetLastError() != cudaSuccess) return set_err(HPX_ERR_CUDA);
    return set_err(HPX_OK);
}

int hpx_healpix_analysis(hpx_plan_s* P, const void* maps, void* alm, int niter) {
    if (!P || !alm || !maps || niter < 0 || niter > 1000) return set_err(HPX_ERR_ARG);
    if (P->group || !(P->flags & HPX_FLAG_JACOBI)) return set_err(HPX_ERR_STATE);
    if ((P->flags & HPX_FLAG_CHECKED) && (!device_pointer(P, maps) || !device_pointer(P, alm)))
        return set_err(HPX_ERR_ARG);
    if (P->precision == HPX_FP64)
        hpx::launch_healpix_jacobi<double>(P, (const double*)maps, (double*)alm, niter, P->stream);
    else
        hpx::launch_healpix_jacobi<float>(P, (const float*)maps, (float*)alm, niter, P->stream);
    if (cudaGetLastError() != cudaSuccess) return set_err(HPX_ERR_CUDA);
    return set_err(HPX_OK);
}

int hpx_set_profiling(hpx_plan_s* P, int enable) {
    if (!P) return set_err(HPX_ERR_ARG);
    if (P->group) return set_err(HPX_ERR_STATE);
    if (enable && !P->ev) {
        const int n = hpx_plan_s::kMaxProf * (hpx_plan_s::kStages + 1);
        P->ev = new (std::nothrow) cudaEvent_t[n];
        if (!P->ev) return set_err(HPX_ERR_OOM);
        for (int k = 0; k < n; ++k)
            if (cudaEventCreate(&P->ev[k]) != cudaSuccess) return set_err(HPX_ERR_CUDA);
    }
    P->prof = enable != 0;
    P->nprof = 0;
    return set_err(HPX_OK);
}

int hpx_stage_times(hpx_plan_s* P, float* ms, int n, int* ncalls) {
    if (!P || !ms || n < hpx_plan_s::kStages) return set_err(HPX_ERR_ARG);
    if (P->group) return set_err(HPX_ERR_STATE);
    for (int k = 0; k < n; ++k) ms[k] = 0.0f;
    for (int c = 0; c < P->nprof; ++c) {
        cudaEvent_t* ev = P->ev + (size_t)c * (hpx_plan_s::kStages + 1);
        if (cudaEventSynchronize(ev[hpx_plan_s::kStages]) != cudaSuccess) return set_err(HPX_ERR_CUDA);
        for (int k = 0; k < hpx_plan_s::kStages; ++k) {
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, ev[k], ev[k + 1]) != cudaSuccess) return set_err(HPX_ERR_CUDA);
            ms[k] += t;
        }
    }
    if (ncalls) *ncalls = P->nprof;
    P->nprof = 0;
    return set_err(HPX_OK);
}

int hpx_cl(hpx_plan_s* P, const void* alm, double* cl) {
    if (!P || !alm || !cl) return set_err(HPX_ERR_ARG);
    if (P->group) return set_err(hpx::group_cl(P, alm, cl));
    if (P->precision == HPX_FP64) hpx::launch_cl<double>(P, (const double*)alm, cl, P->stream);
    else hpx::launch_cl<float>(P, (const float*)alm, cl, P->stream);
    if (cudaGetLastError() != cudaSuccess) return set_err(HPX_ERR_CUDA);
    return set_err(HPX_OK);
}

int hpx_sync(hpx_plan_s* P) {
    if (!P) return set_err(HPX_ERR_ARG);
    if (cudaStreamSynchronize(P->stream) != cudaSuccess) return set_err(HPX_ERR_CUDA);
    // device status words: the plan's own, or those of a group plan's sub-plans
    int first = HPX_OK;
    std::vector<hpx_plan_s*> all{P};
    if (P->group) all.insert(all.end(), P->subs.begin(), P->subs.end());
    for (hpx_plan_s* Q : all) {
        if (!Q->d_status) continue;
        int st = 0;
        if (cudaMemcpy(&st, Q->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return set_err(HPX_ERR_CUDA);
        if (st != 0) {
            cudaMemset(Q->d_status, 0, sizeof(int));
            if (first == HPX_OK) first = st;
        }
    }
    if (first != HPX_OK) return set_err(first);
    if (P->status != 0) return set_err(P->status);
    return set_err(HPX_OK);
}

void hpx_destroy(hpx_plan_s* P) {
    if (!P) return;
    cudaStreamSynchronize(P->stream);
    free_plan(P);
}

int64_t hpx_npix(const hpx_plan_s* P) { return P ? P->g.npix : 0; }
int64_t hpx_nalm(const hpx_plan_s* P) { return P ? P->g.nalm : 0; }
int hpx_plan_lmax(const hpx_plan_s* P) { return P ? P->g.L : -1; }
int64_t hpx_plan_bytes(const hpx_plan_s* P) { return P ? P->bytes : 0; }
int hpx_plan_flags(const hpx_plan_s* P) { return P ? (int)P->flags : -1; }

int hpx_plan_tuning(const hpx_plan_s* P, int* ring_elems, int* fft_elems, int* sweep_form, int* pack_pass,
                    int* ring_form) {
    if (!P || P->group || !ring_elems || !fft_elems || !sweep_form || !pack_pass || !ring_form)
        return set_err(HPX_ERR_ARG);
    *ring_form = P->ringForm;
    *ring_elems = P->ringE;
    *fft_elems = P->latE;
    *sweep_form = P->rotForm;
    *pack_pass = P->packSep;
    return set_err(HPX_OK);
}

int hpx_plan_set_tuning(hpx_plan_s* P, int ring_elems, int fft_elems, int sweep_form, int pack_pass,
                        int ring_form) {
    if (!P || P->group) return set_err(HPX_ERR_ARG);
    auto ok = [](int e) { return e == 16 || e == 32; };
    if (!ok(ring_elems) || !ok(fft_elems) || sweep_form < 0 || sweep_form > 2 || (pack_pass != 0 && pack_pass != 1) ||
        (ring_form != 0 && ring_form != 1))
        return set_err(HPX_ERR_ARG);
    P->ringForm = ring_form;
    P->ringE = ring_elems;
    P->latE = fft_elems;
    P->rotForm = sweep_form;
    P->packSep = pack_pass;
    // captured graphs hold the old launch shapes: capture again on the next call
    for (auto& e : P->graphs) cudaGraphExecDestroy(e.exec);
    P->graphs.clear();
    return set_err(HPX_OK);
}

int hpx_plan_launches(const hpx_plan_s* P) {
    if (!P) return -1;
    if (P->group) {   // the persistent short-ring launches, then each sub-plan's other stages
        int n = (P->nRingLong > 0) + (P->nRingItems > P->nRingLong);
        for (const hpx_plan_s* S : P->subs) {
            n += hpx_plan_launches(S);
            for (const auto& c : S->ringClasses) n -= c.N < hpx::kRingCtMin;   // in the persistent launches
        }
        for (size_t s = 0; s < P->subs.size(); ++s) n += P->sub_inplace[s] ? 0 : 2;   // gather + scatter
        return n;
    }
    int n = P->ringList ? (int)P->ringClasses.size() : 1;   // ring FFTs
    n += 3;                                                 // poles, spreading, grid FFTs
    if (P->flags & HPX_FLAG_CG) n += 1;                     // CG solves
    n += P->fusedM ? 1 : 2;                                 // operators, or D (or C) and the sweeps
    if (P->flags & HPX_FLAG_CHECKED) n += 1;
    return n;
}

int hpx_selftest_timeout(hpx_plan_s* P, int spins) {
    if (!P || spins < 1 || spins > (1 << 20)) return set_err(HPX_ERR_ARG);
    hpx_plan_s* Q = P->group ? P->subs[0] : P;   // a group reports through its sub-plans
    cudaSetDevice(P->device);
    hpx::launch_timeout_selftest(Q, spins, P->stream);
    return set_err(cudaGetLastError() == cudaSuccess ? HPX_OK : HPX_ERR_CUDA);
}

int hpx_last_error(void) { return g_last_error; }

const char* hpx_strerror(int code) {
    switch (code) {
        case HPX_OK: return "ok";
        case HPX_ERR_ARG: return "invalid argument";
        case HPX_ERR_NSIDE: return "nside must be a power of two in [2, 2048] (FP64: [2, 1024])";
        case HPX_ERR_LMAX: return "lmax must satisfy 0 <= lmax <= 2 nside";
        case HPX_ERR_CUDA: return "CUDA runtime error";
        case HPX_ERR_OOM: return "out of device memory";
        case HPX_ERR_TIMEOUT: return "a bounded device-side wait timed out";
        case HPX_ERR_STATE: return "operation not valid for this plan";
        case HPX_ERR_NONFINITE: return "an input held NaN or infinity";
        default: return "unknown error";
    }
}

}  // extern "C"
