// Uneven batches: maps of different nside (or lmax) analysed by one plan.
//
// A group plan holds one uniform sub-plan per distinct (nside, lmax).  The caller's
// maps, coefficients and spectra are concatenated in batch order; a sub-plan
// whose maps are adjacent in the batch works on the caller's arrays in place.
// The others read their maps in place too, through a table of per-map offsets
// (the ring and pole stages), and write their coefficients into a plan-owned
// staging buffer that is scattered back after the launch (segment_copy_kernel);
// the directions that write maps (adjoint, synthesis) stage the maps the same
// way.  The launches start and end on the group's stream, so HPX_FLAG_GRAPH
// captures the whole batch -- every nside -- as one CUDA graph.
#include <algorithm>
#include <map>
#include <new>

#include "../../include/hpx.h"
#include "plan.h"

namespace hpx {

// Copies `count` segments of `seg` bytes (a multiple of 8) between a packed
// staging array and the caller's array, whose segment for batch index idx[k]
// starts at byte off[idx[k]].  gather: caller -> staging; else staging -> caller.
__global__ void segment_copy_kernel(const unsigned char* __restrict__ src, unsigned char* __restrict__ dst,
                                    const int* __restrict__ idx, const int64_t* __restrict__ off, int64_t seg,
                                    bool gather) {
    const int k = blockIdx.y;
    const int64_t caller = off[idx[k]];
    const int64_t packed = (int64_t)k * seg;
    const uint2* s = reinterpret_cast<const uint2*>(src + (gather ? caller : packed));
    uint2* d = reinterpret_cast<uint2*>(dst + (gather ? packed : caller));
    const int64_t n = seg / 8;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        d[e] = s[e];
}

namespace {

void seg_copy(const hpx_plan_s* P, int s, const void* src, void* dst, const int64_t* off, int64_t seg, bool gather,
              cudaStream_t st) {
    dim3 grid((unsigned)std::min<int64_t>((seg / 8 + 255) / 256, 1024), P->sub_count[s]);
    segment_copy_kernel<<<grid, 256, 0, st>>>((const unsigned char*)src, (unsigned char*)dst,
                                              P->d_idx + P->sub_first[s], off, seg, gather);
}
void seg_copy(const hpx_plan_s* P, int s, const void* src, void* dst, const int64_t* off, int64_t seg, bool gather) {
    seg_copy(P, s, src, dst, off, seg, gather, P->stream);
}

// The sub-plans of an analysis run concurrently: each on a stream of its own
// that waits for the group's stream (fork), and the group's stream waits for all
// of them (join).  Under stream capture (HPX_FLAG_GRAPH) this becomes one graph
// with a branch per sub-plan.
void fork(hpx_plan_s* G) { cudaEventRecord(G->sfork, G->stream); }
cudaStream_t branch(hpx_plan_s* G, size_t s) {
    cudaStreamWaitEvent(G->sstreams[s], G->sfork, 0);
    return G->sstreams[s];
}
void join(hpx_plan_s* G) {
    for (size_t s = 0; s < G->subs.size(); ++s) {
        cudaEventRecord(G->sjoin[s], G->sstreams[s]);
        cudaStreamWaitEvent(G->stream, G->sjoin[s], 0);
    }
}

int64_t nalm_of(int L) { return (int64_t)(L + 1) * (L + 2) / 2; }

}  // namespace

hpx_plan_s* group_create(const hpx_plan_desc* d, int* err) {
    *err = HPX_ERR_ARG;
    const int B = d->batch;
    const bool fp64 = d->precision == HPX_FP64;
    // nside and lmax of map i
    auto nside_of = [&](int i) { return d->nsides ? d->nsides[i] : d->nside; };
    auto lmax_of = [&](int i) {
        const int l = d->lmaxs ? d->lmaxs[i] : d->lmax;
        return l < 0 ? 2 * nside_of(i) : l;
    };
    for (int i = 0; i < B; ++i) {
        const int ns = nside_of(i);
        if (ns < 2 || (ns & (ns - 1)) || ns > (fp64 ? 1024 : 2048)) { *err = HPX_ERR_NSIDE; return nullptr; }
        const int l = d->lmaxs ? d->lmaxs[i] : d->lmax;
        if (l < -1 || lmax_of(i) > 2 * ns) { *err = HPX_ERR_LMAX; return nullptr; }
    }
    hpx_plan_s* G = new (std::nothrow) hpx_plan_s();
    if (!G) { *err = HPX_ERR_OOM; return nullptr; }
    G->group = true;
    G->precision = d->precision;
    G->flags = d->flags;
    G->stream = nullptr;
    cudaGetDevice(&G->device);
    const size_t es = fp64 ? 8 : 4;
    // per-map offsets (bytes) in the caller's concatenated arrays
    std::vector<int64_t> mapoff(B), almoff(B), cloff(B), almel(B), clel(B);
    std::vector<int> lmaxv(B);
    std::map<std::pair<int, int>, std::vector<int>> byNside;   // (nside, lmax) -> maps
    int64_t om = 0, oa = 0, oc = 0;
    int Lmax_all = 0;
    for (int i = 0; i < B; ++i) {
        const int ns = nside_of(i);
        const int L = lmax_of(i);
        Lmax_all = std::max(Lmax_all, L);
        mapoff[i] = om * (int64_t)es;
        almoff[i] = oa * (int64_t)es * 2;
        cloff[i] = oc * 8;
        almel[i] = oa;
        clel[i] = oc;
        lmaxv[i] = L;
        om += 12LL * ns * ns;
        oa += nalm_of(L);
        oc += L + 1;
        byNside[{ns, L}].push_back(i);
    }
    G->total_npix = om;
    if (cudaEventCreateWithFlags(&G->sfork, cudaEventDisableTiming) != cudaSuccess) {
        *err = HPX_ERR_CUDA;
        delete G;
        return nullptr;
    }
    G->total_nalm = oa;
    G->total_ncl = oc;
    G->g = Geometry{};
    G->g.L = Lmax_all;
    G->g.B = B;
    G->g.npix = om;
    G->g.nalm = oa;
    std::vector<int> idx;
    bool ok = true;
    for (auto& kv : byNside) {
        const int ns = kv.first.first;
        const std::vector<int>& maps = kv.second;
        hpx_plan_desc sd = *d;
        sd.nside = ns;
        sd.lmax = kv.first.second;
        sd.batch = (int)maps.size();
        // the group checks its inputs itself; sub-plans get the rest of the flags
        sd.flags = d->flags & ~(unsigned)(HPX_FLAG_GRAPH | HPX_FLAG_CHECKED);
        sd.nsides = nullptr;
        sd.lmaxs = nullptr;
        hpx_plan_s* S = hpx_plan_ex(&sd);
        if (!S) { *err = hpx_last_error(); ok = false; break; }
        G->subs.push_back(S);
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            *err = HPX_ERR_CUDA;
            ok = false;
        }
        G->sstreams.push_back(st);
        G->sjoin.push_back(ev);
        if (!ok) break;
        G->bytes += S->bytes;
        G->sub_count.push_back((int)maps.size());
        G->sub_first.push_back((int)idx.size());
        bool adj = true;
        for (size_t k = 1; k < maps.size(); ++k) adj = adj && maps[k] == maps[k - 1] + 1;
        G->sub_inplace.push_back(adj ? 1 : 0);
        G->sub_mapoff.push_back(mapoff[maps[0]]);
        G->sub_almoff.push_back(almoff[maps[0]]);
        G->sub_cloff.push_back(cloff[maps[0]]);
        void *sm = nullptr, *sa = nullptr, *sc = nullptr;
        if (!adj) {
            const size_t nm = maps.size();
            if (cudaMalloc(&sm, nm * S->g.npix * es) != cudaSuccess ||
                cudaMalloc(&sa, nm * S->g.nalm * es * 2) != cudaSuccess ||
                cudaMalloc(&sc, nm * (S->g.L + 1) * 8) != cudaSuccess) {
                *err = HPX_ERR_OOM;
                ok = false;
            }
            G->bytes += (int64_t)(nm * (S->g.npix * es + S->g.nalm * es * 2 + (S->g.L + 1) * 8));
        }
        G->stage_maps.push_back(sm);
        G->stage_alm.push_back(sa);
        G->stage_cl.push_back(sc);
        if (!ok) break;
        idx.insert(idx.end(), maps.begin(), maps.end());
    }
    if (ok) {
        ok = cudaMalloc(&G->d_idx, idx.size() * sizeof(int)) == cudaSuccess &&
             cudaMalloc(&G->d_mapoff, B * sizeof(int64_t)) == cudaSuccess &&
             cudaMalloc(&G->d_almoff, B * sizeof(int64_t)) == cudaSuccess &&
             cudaMalloc(&G->d_cloff, B * sizeof(int64_t)) == cudaSuccess &&
             cudaMalloc(&G->d_almel, B * sizeof(int64_t)) == cudaSuccess &&
             cudaMalloc(&G->d_clel, B * sizeof(int64_t)) == cudaSuccess &&
             cudaMalloc(&G->d_lmax, B * sizeof(int)) == cudaSuccess;
        if (ok) {
            cudaMemcpy(G->d_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice);
            cudaMemcpy(G->d_mapoff, mapoff.data(), B * sizeof(int64_t), cudaMemcpyHostToDevice);
            cudaMemcpy(G->d_almoff, almoff.data(), B * sizeof(int64_t), cudaMemcpyHostToDevice);
            cudaMemcpy(G->d_cloff, cloff.data(), B * sizeof(int64_t), cudaMemcpyHostToDevice);
            cudaMemcpy(G->d_almel, almel.data(), B * sizeof(int64_t), cudaMemcpyHostToDevice);
            cudaMemcpy(G->d_clel, clel.data(), B * sizeof(int64_t), cudaMemcpyHostToDevice);
            cudaMemcpy(G->d_lmax, lmaxv.data(), B * sizeof(int), cudaMemcpyHostToDevice);
        } else {
            *err = HPX_ERR_OOM;
        }
    }
    // per-map element offsets of the sub-plans whose maps are not adjacent: the
    // analysis reads their maps in place through them
    for (size_t s = 0; ok && s < G->subs.size(); ++s) {
        if (G->sub_inplace[s]) continue;
        std::vector<int64_t> offs(G->sub_count[s]);
        for (int k = 0; k < G->sub_count[s]; ++k) offs[k] = mapoff[idx[G->sub_first[s] + k]] / (int64_t)es;
        hpx_plan_s* S = G->subs[s];
        ok = cudaMalloc(&S->mapIdx, offs.size() * sizeof(int64_t)) == cudaSuccess &&
             cudaMemcpy(S->mapIdx, offs.data(), offs.size() * sizeof(int64_t), cudaMemcpyHostToDevice) == cudaSuccess;
        if (!ok) *err = HPX_ERR_OOM;
    }
    if (!ok) {
        group_free(G);
        return nullptr;
    }
    *err = HPX_OK;
    return G;
}

void group_free(hpx_plan_s* G) {
    for (cudaStream_t st : G->sstreams)
        if (st) cudaStreamSynchronize(st);
    for (hpx_plan_s* S : G->subs) hpx_destroy(S);
    for (cudaStream_t st : G->sstreams)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : G->sjoin)
        if (ev) cudaEventDestroy(ev);
    if (G->sfork) cudaEventDestroy(G->sfork);
    if (G->ringJobs) cudaFree(G->ringJobs);
    if (G->ringItems) cudaFree(G->ringItems);
    if (G->ringEv) cudaEventDestroy(G->ringEv);
    for (void* q : G->stage_maps) if (q) cudaFree(q);
    for (void* q : G->stage_alm) if (q) cudaFree(q);
    for (void* q : G->stage_cl) if (q) cudaFree(q);
    if (G->d_idx) cudaFree(G->d_idx);
    if (G->d_mapoff) cudaFree(G->d_mapoff);
    if (G->d_almoff) cudaFree(G->d_almoff);
    if (G->d_cloff) cudaFree(G->d_cloff);
    if (G->d_almel) cudaFree(G->d_almel);
    if (G->d_clel) cudaFree(G->d_clel);
    if (G->d_lmax) cudaFree(G->d_lmax);
}

// An uneven analysis: the gathers of the sub-plans whose maps are not adjacent,
// then the ring stage of every map of every Nside in one persistent launch (the
// work list of build_ring_list), then the remaining stages of each sub-plan as
// concurrent branches, each ending with its scatter.
int group_analyze(hpx_plan_s* G, const void* maps, void* alm) {
    const size_t es = G->precision == HPX_FP64 ? 8 : 4;
    fork(G);
    // the short rings of every sub-plan on the group's stream, meanwhile each
    // branch runs its sub-plan's compile-time ring classes
    if (G->precision == HPX_FP64)
        launch_ring_list<double>((const RingJob<double>*)G->ringJobs, G->ringItems, G->nRingItems, G->nRingLong,
                                 (const double*)maps, G->stream);
    else
        launch_ring_list<float>((const RingJob<float>*)G->ringJobs, G->ringItems, G->nRingItems, G->nRingLong,
                                (const float*)maps, G->stream);
    cudaEventRecord(G->ringEv, G->stream);
    int rc = HPX_OK;
    for (size_t s = 0; s < G->subs.size() && rc == HPX_OK; ++s) {
        hpx_plan_s* S = G->subs[s];
        const cudaStream_t st = branch(G, s);
        hpx_set_stream(S, st);
        // maps read in place: adjacent ones from the sub-plan's first map, the
        // others through the sub-plan's per-map offsets from the caller's base
        const void* smaps = G->sub_inplace[s] ? (const void*)((const unsigned char*)maps + G->sub_mapoff[s]) : maps;
        if (G->precision == HPX_FP64) launch_ring_fft<double>(S, (const double*)smaps, st, 0.0, kRingCtMin);
        else launch_ring_fft<float>(S, (const float*)smaps, st, 0.f, kRingCtMin);
        cudaStreamWaitEvent(st, G->ringEv, 0);
        if (G->sub_inplace[s]) {
            rc = analyze_after_rings(S, (const unsigned char*)maps + G->sub_mapoff[s],
                                     (unsigned char*)alm + G->sub_almoff[s]);
        } else {
            rc = analyze_after_rings(S, maps, G->stage_alm[s]);
            if (rc == HPX_OK)
                seg_copy(G, (int)s, G->stage_alm[s], alm, G->d_almoff, S->g.nalm * (int64_t)es * 2, false, st);
        }
    }
    join(G);   // also after an error: every branch rejoins the group's stream
    if (rc != HPX_OK) return rc;
    return cudaGetLastError() == cudaSuccess ? HPX_OK : HPX_ERR_CUDA;
}

namespace {
// alm -> maps through every sub-plan with `fn` (the adjoint or the SH synthesis)
int group_alm_to_maps(hpx_plan_s* G, const void* alm, void* maps, int (*fn)(hpx_plan_s*, const void*, void*)) {
    for (size_t s = 0; s < G->subs.size(); ++s) {
        hpx_plan_s* S = G->subs[s];
        hpx_set_stream(S, G->stream);
        const size_t es = G->precision == HPX_FP64 ? 8 : 4;
        if (G->sub_inplace[s]) {
            const int rc = fn(S, (const unsigned char*)alm + G->sub_almoff[s], (unsigned char*)maps + G->sub_mapoff[s]);
            if (rc != HPX_OK) return rc;
        } else {
            seg_copy(G, (int)s, alm, G->stage_alm[s], G->d_almoff, S->g.nalm * (int64_t)es * 2, true);
            const int rc = fn(S, G->stage_alm[s], G->stage_maps[s]);
            if (rc != HPX_OK) return rc;
            seg_copy(G, (int)s, G->stage_maps[s], maps, G->d_mapoff, S->g.npix * (int64_t)es, false);
        }
    }
    return cudaGetLastError() == cudaSuccess ? HPX_OK : HPX_ERR_CUDA;
}
}  // namespace

int group_synthesize(hpx_plan_s* G, const void* alm, void* maps) { return group_alm_to_maps(G, alm, maps, hpx_synthesize); }

int group_analyze_vjp(hpx_plan_s* G, const void* galm, void* gmaps) {
    return group_alm_to_maps(G, galm, gmaps, hpx_analyze_vjp);
}

int group_sh_synthesis(hpx_plan_s* G, const void* alm, void* maps) {
    return group_alm_to_maps(G, alm, maps, hpx_sh_synthesis);
}

// every map of the batch in one launch, located through the per-map tables
int group_cl(hpx_plan_s* G, const void* alm, double* cl) {
    if (G->precision == HPX_FP64) launch_cl<double>(G, (const double*)alm, cl, G->stream);
    else launch_cl<float>(G, (const float*)alm, cl, G->stream);
    return cudaGetLastError() == cudaSuccess ? HPX_OK : HPX_ERR_CUDA;
}

namespace {
// The work list of the persistent ring kernel: (sub-plan, ring pair, map) for
// every map of the batch, longest transforms first, and the job table of the
// sub-plans (their tables, Y workspaces and where their maps are).
template <class T>
bool build_ring_list(hpx_plan_s* G) {
    const size_t es = sizeof(T);
    std::vector<RingJob<T>> jobs;
    struct Item {
        int len, s, i, b;
    };
    std::vector<Item> items;
    for (size_t s = 0; s < G->subs.size(); ++s) {
        const hpx_plan_s* S = G->subs[s];
        const auto& t = S->t;
        RingJob<T> J;
        J.mapoff = G->sub_inplace[s] ? G->sub_mapoff[s] / (int64_t)es : 0;
        J.mapIdx = S->mapIdx;
        J.Y = (cplx<T>*)S->Y;
        J.nphi = t.nphi; J.startN = t.startN; J.startS = t.startS; J.pow2 = t.pow2; J.logn = t.logn;
        J.fftL = t.fftL; J.logL = t.logL; J.shifted = t.shifted;
        J.shOff = t.shOff; J.chOff = t.chOff; J.bhOff = t.bhOff;
        J.shift = (const cplx<T>*)t.shift; J.chirp = (const cplx<T>*)t.chirp; J.bhat = (const cplx<T>*)t.bhat;
        J.tw = (const cplx<T>*)t.twid;
        J.twlen = S->g.Lmax; J.p = S->g.p; J.Q = S->g.Q; J.L = S->g.L; J.npix = S->g.npix;
        jobs.push_back(J);
        // transform length of every ring pair, from the host copy of the geometry
        const int ns = S->g.ns;
        for (int i = 0; i < S->g.npairs; ++i) {
            const int j = i + 1;
            const int n = (j < ns) ? 4 * j : 4 * ns;
            int len = n;
            if (n & (n - 1)) {   // Bluestein: the power of two >= 2 n - 1
                len = 1;
                while (len < 2 * n - 1) len <<= 1;
            }
            if (len >= kRingCtMin) continue;   // the sub-plan's compile-time kernels
            for (int b = 0; b < G->sub_count[s]; ++b) items.push_back({len, (int)s, i, b});
        }
    }
    std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return a.len > b.len; });
    std::vector<int4> packed(items.size());
    for (size_t k = 0; k < items.size(); ++k) packed[k] = make_int4(items[k].s, items[k].i, items[k].b, items[k].len);
    if (cudaMalloc(&G->ringJobs, jobs.size() * sizeof(RingJob<T>)) != cudaSuccess ||
        cudaMalloc(&G->ringItems, packed.size() * sizeof(int4)) != cudaSuccess)
        return false;
    cudaMemcpy(G->ringJobs, jobs.data(), jobs.size() * sizeof(RingJob<T>), cudaMemcpyHostToDevice);
    cudaMemcpy(G->ringItems, packed.data(), packed.size() * sizeof(int4), cudaMemcpyHostToDevice);
    G->nRingItems = (int)packed.size();
    G->nRingLong = 0;
    while (G->nRingLong < (int)items.size() && items[G->nRingLong].len > 512) ++G->nRingLong;
    return cudaEventCreateWithFlags(&G->ringEv, cudaEventDisableTiming) == cudaSuccess;
}
}  // namespace

bool group_build_ring_list(hpx_plan_s* G) {
    return G->precision == HPX_FP64 ? build_ring_list<double>(G) : build_ring_list<float>(G);
}

}  // namespace hpx
