// Batch of independent periodic boxes stepped together (the batched-ensemble
// workload): uneven boxes, each with its own extents, cell size, shape order,
// particles and fields, all with one time step.
//
// Layout.  One pooled context holds every box: the particles of all boxes in
// one double-buffered SoA, the nine field components as arrays over all
// boxes' cells (box b at cells [cbase_b, cbase_b + C_b)), one sort over all
// boxes (each box starts on a multiple of 64 cells, the gaps stay zero and
// hold no keys).  Cell keys carry the box's first key as a base, so the counting sort
// groups particles by box and then by tile, and box b's particles always sit
// at [pbase_b, pbase_b + N_b).  A per-box view context (pointers offset into
// the pool) serves loading, getters and diagnostics with the single-box code.
//
// Step.  Sort (at the cadence), then per shape order one persistent tile
// kernel whose CTAs pull (box, tile) items heaviest first from a queue, its
// outsider kernel, and the Yee update of all boxes (a block table maps blocks
// to boxes).  pic_batch_step captures its whole step loop into one CUDA graph
// and replays it.  An autotuner times tile shape x particles per lane run x
// sort cadence from a stored state and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pic_ctx.h"
#include "pic_step_common.cuh"

namespace pic {
void set_last_error(const std::string& msg);
}

namespace {

pic_status bfail(pic_status s, const std::string& msg) {
    pic::set_last_error(msg);
    return s;
}

pic_status bcuda(cudaError_t e, const char* where) {
    cudaGetLastError();
    return bfail(PIC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define BCUDA(call)                                    \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return bcuda(e_, #call); \
    } while (0)

struct BoxInfo {
    int n[3];
    double d[3];
    int order;
    int64_t cbase, C;
    int64_t pbase = 0, np = 0;
    double w_max = 0.0;
    pic::Geom g;
};

struct ClassInfo {
    int order;
    int nitems;
    size_t items_off;     // byte offset of the items in the table block
    int64_t outl_off;     // first slot of this class's outsider list
};

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

}  // namespace

struct pic_batch {
    pic_ctx pool;
    std::vector<BoxInfo> box;
    std::vector<ClassInfo> cls;
    pic_batch_tuning tune{{8, 8, 8}, 0, 1};
    bool loaded = false;
    int sms = 152;
    // device tables (one allocation): StepArgs per box for both buffer roles,
    // YeeArgs (h = dt/2, h = dt), Yee block map, work items, pbase, counters
    char* tab = nullptr;
    size_t tab_bytes = 0;
    size_t off_args[2] = {0, 0}, off_yb = 0, off_ye = 0, off_blocks = 0, off_pbase = 0, off_counters = 0;
    size_t off_maps = 0;          // one E/B TMA descriptor per box
    std::vector<char> map_ok;     // per box: its descriptor is valid
    int nblocks = 0;
    // captured step loop
    cudaGraphExec_t graph = nullptr;
    int g_steps = 0, g_cur = 0, g_since = 0, g_end_cur = 0, g_end_since = 0;
    int64_t g_kernels = 0;
    uint64_t version = 1, g_version = 0;
    int64_t launches = 0;
    bool own_stream = false;
};

namespace {

// Geometry of box b with tiles no larger than `tile` (powers of two dividing the extents).
pic::Geom box_geom(const BoxInfo& B, const int tile[3]) {
    pic::Geom g;
    int64_t C = 1;
    for (int a = 0; a < 3; ++a) {
        int T = 1;
        while (T * 2 <= tile[a] && B.n[a] % (T * 2) == 0) T *= 2;
        g.n[a] = B.n[a];
        g.d[a] = B.d[a];
        g.L[a] = B.n[a] * B.d[a];
        g.T[a] = T;
        g.lT[a] = ilog2(T);
        g.nt[a] = B.n[a] / T;
        C *= B.n[a];
    }
    g.cpt = g.T[0] * g.T[1] * g.T[2];
    g.C = C;
    g.ntiles = int64_t(g.nt[0]) * g.nt[1] * g.nt[2];
    g.kbase = int(B.cbase);
    g.zopen = 0;
    return g;
}

// Single-box view of box i: pointers into the pool, the box's geometry and weight scale.
pic_ctx make_view(const pic_batch* b, int i) {
    const BoxInfo& B = b->box[size_t(i)];
    const pic_ctx& P = b->pool;
    pic_ctx v;
    v.g = B.g;
    v.dt = P.dt;
    v.prec = P.prec;
    v.order = B.order;
    v.sort_every = b->tune.sort_every;
    v.stream = P.stream;
    v.device = P.device;
    v.rsize = P.rsize;
    for (int c = 0; c < 9; ++c) v.F[c] = static_cast<char*>(P.F[c]) + B.cbase * P.rsize;
    v.np = v.cap = B.np;
    v.q = P.q;
    v.m = P.m;
    v.w_max = B.w_max;
    for (int r = 0; r < 2; ++r) {
        for (int a = 0; a < 7; ++a) v.P[r].a[a] = static_cast<char*>(P.P[r].a[a]) + B.pbase * P.rsize;
        v.P[r].key = P.P[r].key + B.pbase;
        v.P[r].id = P.P[r].id + B.pbase;
    }
    v.cur = P.cur;
    v.err = P.err;
    v.d_step = P.d_step;
    v.dsum = P.dsum;
    v.stage = P.stage;
    v.sms = b->sms;
    v.step = P.step;
    return v;
}

template <typename R> void fill_args(const pic_batch* b, std::vector<char>& host) {
    const size_t nb = b->box.size();
    const pic_ctx& P = b->pool;
    for (int r = 0; r < 2; ++r) {
        auto* args = reinterpret_cast<pic::StepArgs<R>*>(host.data() + b->off_args[r]);
        for (size_t i = 0; i < nb; ++i) {
            pic_ctx v = make_view(b, int(i));
            v.cur = r;
            pic::StepArgs<R> A = pic::make_args<R>(&v);
            // the tile kernel indexes particles globally (offsets of the pooled sort)
            for (int a = 0; a < 7; ++a) {
                A.pa[a] = static_cast<R*>(P.P[r].a[a]);
                A.spa[a] = A.pa[a];
            }
            A.key = P.P[r].key;
            A.skey = A.key;  // in place: the source is the pooled buffer itself
            A.sid = A.did = P.P[r].id;
            A.offsets = P.offsets + b->box[i].cbase;
            A.np = P.np;
            A.run = b->tune.run;
            int k = 0;
            while (b->cls[size_t(k)].order != b->box[i].order) ++k;
            int* counters = reinterpret_cast<int*>(b->tab + b->off_counters);
            A.outn = counters + 4 + k;
            A.outl = P.outl + b->cls[size_t(k)].outl_off;
            A.tmap = b->map_ok.size() > i && b->map_ok[i]
                         ? reinterpret_cast<const CUtensorMap*>(b->tab + b->off_maps) + i
                         : nullptr;
            args[i] = A;
        }
    }
    auto* yb = reinterpret_cast<pic::YeeArgs<R>*>(host.data() + b->off_yb);
    auto* ye = reinterpret_cast<pic::YeeArgs<R>*>(host.data() + b->off_ye);
    for (size_t i = 0; i < nb; ++i) {
        const BoxInfo& B = b->box[i];
        pic::YeeArgs<R> Y;
        for (int d = 0; d < 3; ++d) {
            Y.E[d] = reinterpret_cast<R*>(static_cast<char*>(P.F[d]) + B.cbase * sizeof(R));
            Y.B[d] = reinterpret_cast<R*>(static_cast<char*>(P.F[3 + d]) + B.cbase * sizeof(R));
            Y.J[d] = reinterpret_cast<const R*>(static_cast<char*>(P.F[6 + d]) + B.cbase * sizeof(R));
            Y.n[d] = B.n[d];
            Y.inv[d] = R(1.0 / B.d[d]);
        }
        Y.step = nullptr;
        Y.zopen = 0;
        Y.ckc = 0;
        Y.h = R(0.5 * P.dt);
        yb[i] = Y;
        Y.h = R(P.dt);
        ye[i] = Y;
    }
}

// (Re)build and upload every device table for the current tuning and load.
pic_status build_tables(pic_batch* b) {
    const size_t nb = b->box.size();
    const size_t rs = b->pool.rsize;
    const size_t args_sz = rs == 8 ? sizeof(pic::StepArgs<double>) : sizeof(pic::StepArgs<float>);
    const size_t yee_sz = rs == 8 ? sizeof(pic::YeeArgs<double>) : sizeof(pic::YeeArgs<float>);
    auto align = [](size_t v) { return (v + 255) & ~size_t(255); };
    // classes by shape order; items heaviest first (particles per tile), then box, tile
    b->cls.clear();
    for (int order = 3; order >= 1; --order) {
        bool any = false;
        for (const auto& B : b->box)
            if (B.order == order) any = true;
        if (!any) continue;
        int64_t before = 0;
        for (const auto& c : b->cls)
            for (const auto& B : b->box)
                if (B.order == c.order) before += B.np;
        b->cls.push_back({order, 0, 0, before});
    }
    std::vector<std::vector<int2>> items(b->cls.size());
    for (size_t k = 0; k < b->cls.size(); ++k) {
        std::vector<std::pair<double, int2>> w;
        for (size_t i = 0; i < nb; ++i) {
            const BoxInfo& B = b->box[i];
            if (B.order != b->cls[k].order) continue;
            const double load = double(B.np) / double(B.g.ntiles);
            for (int64_t t = 0; t < B.g.ntiles; ++t) w.push_back({load, make_int2(int(i), int(t))});
        }
        std::stable_sort(w.begin(), w.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
        for (auto& e : w) items[k].push_back(e.second);
        b->cls[k].nitems = int(items[k].size());
    }
    std::vector<int4> blocks;
    for (size_t i = 0; i < nb; ++i)
        for (int64_t s = 0; s < b->box[i].C; s += pic::kBlock)
            blocks.push_back(make_int4(int(i), int(s), int(std::min<int64_t>(pic::kBlock, b->box[i].C - s)), 0));
    b->nblocks = int(blocks.size());
    size_t off = 0;
    b->off_args[0] = off;
    off = align(off + nb * args_sz);
    b->off_args[1] = off;
    off = align(off + nb * args_sz);
    b->off_yb = off;
    off = align(off + nb * yee_sz);
    b->off_ye = off;
    off = align(off + nb * yee_sz);
    b->off_blocks = off;
    off = align(off + blocks.size() * sizeof(int4));
    for (size_t k = 0; k < b->cls.size(); ++k) {
        b->cls[k].items_off = off;
        off = align(off + items[k].size() * sizeof(int2));
    }
    b->off_pbase = off;
    off = align(off + (nb + 1) * sizeof(int64_t));
    b->off_counters = off;
    off = align(off + 8 * sizeof(int));
    b->off_maps = off;
    off = align(off + nb * sizeof(CUtensorMap));
    if (off > b->tab_bytes) {
        if (b->tab) cudaFree(b->tab);
        b->tab = nullptr;
        b->tab_bytes = 0;
        cudaError_t e = cudaMalloc(&b->tab, off);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? bfail(PIC_ERR_OOM, "batch tables") : bcuda(e, "batch tables");
        b->tab_bytes = off;
    }
    std::vector<char> host(off, 0);
    // each box's E/B (at its cell base in the pool, components one pool apart)
    // as a TMA descriptor for the 8x8x8 layout
    b->map_ok.assign(nb, 0);
    for (size_t i = 0; i < nb; ++i) {
        const BoxInfo& B = b->box[i];
        const void* base = static_cast<const char*>(b->pool.F[0]) + B.cbase * rs;
        auto* m = reinterpret_cast<CUtensorMap*>(host.data() + b->off_maps) + i;
        b->map_ok[i] = pic::encode_eb_tensor_map(m, base, B.n, b->pool.g.C, 0, b->pool.prec) ? 1 : 0;
    }
    if (rs == 8) fill_args<double>(b, host);
    else fill_args<float>(b, host);
    std::memcpy(host.data() + b->off_blocks, blocks.data(), blocks.size() * sizeof(int4));
    for (size_t k = 0; k < b->cls.size(); ++k)
        std::memcpy(host.data() + b->cls[k].items_off, items[k].data(), items[k].size() * sizeof(int2));
    auto* pb = reinterpret_cast<int64_t*>(host.data() + b->off_pbase);
    for (size_t i = 0; i < nb; ++i) pb[i] = b->box[i].pbase;
    pb[nb] = b->pool.np;
    BCUDA(cudaMemcpy(b->tab, host.data(), off, cudaMemcpyHostToDevice));
    b->version += 1;
    return PIC_OK;
}

cudaError_t batch_sort(pic_batch* b) {
    cudaError_t e;
    if ((e = pic::launch_hist(&b->pool)) != cudaSuccess) return e;
    if ((e = pic::launch_scan(&b->pool)) != cudaSuccess) return e;
    if ((e = pic::launch_scatter(&b->pool)) != cudaSuccess) return e;
    b->pool.cur = 1 - b->pool.cur;
    b->pool.since_sort = 0;
    b->pool.sorted = true;
    return cudaSuccess;
}

// Queue nsteps steps; advances the host-side state (cur, since_sort, step).
cudaError_t enqueue_steps(pic_batch* b, int nsteps, int64_t* kernels) {
    pic_ctx& P = b->pool;
    int* counters = reinterpret_cast<int*>(b->tab + b->off_counters);
    for (int s = 0; s < nsteps; ++s) {
        cudaError_t e;
        if (P.since_sort >= b->tune.sort_every) {
            if ((e = batch_sort(b)) != cudaSuccess) return e;
            *kernels += 3;
        }
        if ((e = cudaMemsetAsync(P.F[6], 0, 3 * size_t(P.g.C) * P.rsize, P.stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(counters, 0, 8 * sizeof(int), P.stream)) != cudaSuccess) return e;
        for (size_t k = 0; k < b->cls.size(); ++k) {
            pic::BatchTileLaunch L;
            L.order = b->cls[k].order;
            L.boxes = b->tab + b->off_args[P.cur];
            L.items = reinterpret_cast<const int2*>(b->tab + b->cls[k].items_off);
            L.nitems = b->cls[k].nitems;
            L.queue = counters + k;
            L.pbase = reinterpret_cast<const int64_t*>(b->tab + b->off_pbase);
            L.nboxes = int(b->box.size());
            L.outn = counters + 4 + k;
            L.outl = P.outl + b->cls[k].outl_off;
            L.grid = b->sms;
            if ((e = pic::launch_tile_step_batch(P.prec, L, P.stream)) != cudaSuccess) return e;
            *kernels += L.nitems > 0 ? 2 : 0;
        }
        if ((e = pic::launch_yee_batch(P.prec, b->tab + b->off_yb, b->tab + b->off_ye,
                                       reinterpret_cast<const int4*>(b->tab + b->off_blocks), b->nblocks, P.d_step,
                                       P.stream)) != cudaSuccess)
            return e;
        *kernels += 3;
        P.since_sort += 1;
        P.step += 1;
    }
    return cudaSuccess;
}

void drop_graph(pic_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->g_version = 0;
}

// A graph of nsteps steps from the current (cur, since_sort) state.
pic_status ensure_graph(pic_batch* b, int nsteps) {
    pic_ctx& P = b->pool;
    if (b->graph && b->g_version == b->version && b->g_steps == nsteps && b->g_cur == P.cur &&
        b->g_since == P.since_sort)
        return PIC_OK;
    drop_graph(b);
    const int cur0 = P.cur, since0 = P.since_sort;
    const int64_t step0 = P.step;
    const bool sorted0 = P.sorted;
    int64_t kernels = 0;
    BCUDA(cudaStreamBeginCapture(P.stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = enqueue_steps(b, nsteps, &kernels);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(P.stream, &graph);
    b->g_end_cur = P.cur;
    b->g_end_since = P.since_sort;
    P.cur = cur0;
    P.since_sort = since0;
    P.step = step0;
    P.sorted = sorted0;
    if (e1 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return bcuda(e1, "batch step capture");
    }
    if (e2 != cudaSuccess) return bcuda(e2, "batch end capture");
    cudaError_t e3 = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) {
        b->graph = nullptr;
        return bcuda(e3, "batch graph instantiate");
    }
    b->g_steps = nsteps;
    b->g_cur = cur0;
    b->g_since = since0;
    b->g_kernels = kernels;
    b->g_version = b->version;
    return PIC_OK;
}

cudaError_t launch_graph(pic_batch* b) {
    cudaError_t e = cudaGraphLaunch(b->graph, b->pool.stream);
    if (e != cudaSuccess) return e;
    b->pool.cur = b->g_end_cur;
    b->pool.since_sort = b->g_end_since;
    b->pool.step += b->g_steps;
    b->pool.sorted = true;
    b->launches += b->g_kernels;
    return cudaSuccess;
}

pic_status read_error(pic_batch* b) {
    unsigned hw[4];
    BCUDA(cudaMemcpyAsync(hw, b->pool.err, sizeof(hw), cudaMemcpyDeviceToHost, b->pool.stream));
    BCUDA(cudaStreamSynchronize(b->pool.stream));
    if (hw[0] == 0) return PIC_OK;
    BCUDA(cudaMemsetAsync(b->pool.err, 0, sizeof(hw), b->pool.stream));
    BCUDA(cudaStreamSynchronize(b->pool.stream));
    if (hw[0] & pic::ERRBIT_CHECK) {
        char buf[160];
        std::snprintf(buf, sizeof(buf), "self-check failed at site %u, value 0x%08x%08x", hw[1], hw[3], hw[2]);
        return bfail(PIC_ERR_STATE, buf);
    }
    if (hw[0] & pic::ERRBIT_TIMEOUT) return bfail(PIC_ERR_TIMEOUT, "a bounded device-side wait ran out");
    if (hw[0] & pic::ERRBIT_RANGE) return bfail(PIC_ERR_STATE, "a particle cell key was out of range");
    return bfail(PIC_ERR_PARTICLE, "a particle became non-finite or moved a cell or more in one step");
}

bool valid_tuning(const pic_batch_tuning& t) {
    for (int a = 0; a < 3; ++a)
        if (!is_pow2(t.tile[a]) || t.tile[a] > 8) return false;
    return t.run >= 0 && t.run <= 64 && t.sort_every >= 1 && t.sort_every <= 64;
}

// Switch to tuning t.  With `rekey`, the particle keys are converted from the
// current tile shape and the particles re-sorted; without, the keys are
// taken to be in t's shape already (a state stored under t was restored).
pic_status apply_tuning(pic_batch* b, const pic_batch_tuning& t, bool rekey) {
    std::vector<pic::Geom> old;
    for (auto& B : b->box) old.push_back(B.g);
    b->tune = t;
    for (auto& B : b->box) B.g = box_geom(B, t.tile);
    if (!b->loaded) return PIC_OK;
    if (rekey) {
        for (size_t i = 0; i < b->box.size(); ++i) {
            const BoxInfo& B = b->box[i];
            BCUDA(pic::launch_rekey(b->pool.P[b->pool.cur].key + B.pbase, B.np, old[i], B.g, b->pool.stream));
            b->launches += B.np > 0 ? 1 : 0;
        }
        BCUDA(batch_sort(b));
        b->launches += 3;
    }
    drop_graph(b);
    return build_tables(b);
}

pic_status check_batch(pic_batch* b) { return b ? PIC_OK : bfail(PIC_ERR_ARG, "null batch"); }

pic_status check_box(pic_batch* b, int32_t box) {
    if (pic_status s = check_batch(b)) return s;
    if (box < 0 || box >= int32_t(b->box.size())) return bfail(PIC_ERR_ARG, "box index out of range");
    if (!b->loaded) return bfail(PIC_ERR_STATE, "no particles loaded");
    return PIC_OK;
}

}  // namespace

extern "C" {

pic_status pic_batch_init(int32_t nboxes, const int32_t* n, const double* d, const int32_t* order, double dt,
                          double cfl, int32_t precision, void* cuda_stream, pic_batch** out) {
    if (!out) return bfail(PIC_ERR_ARG, "NULL output");
    *out = nullptr;
    if (nboxes < 1 || !n || !order) return bfail(PIC_ERR_ARG, "need nboxes >= 1, extents and orders");
    if (precision != PIC_FP64 && precision != PIC_FP32_MIXED) return bfail(PIC_ERR_ARG, "unknown precision");
    std::vector<BoxInfo> boxes(static_cast<size_t>(nboxes));
    int64_t C = 0;
    double dt_lim = INFINITY;
    for (int i = 0; i < nboxes; ++i) {
        BoxInfo& B = boxes[size_t(i)];
        B.order = order[i];
        if (B.order < 1 || B.order > 3) return bfail(PIC_ERR_ARG, "order must be 1, 2 or 3");
        double s = 0.0;
        for (int a = 0; a < 3; ++a) {
            B.n[a] = n[3 * i + a];
            B.d[a] = d ? d[3 * i + a] : 1.0;
            if (B.n[a] < B.order + 2 || B.n[a] < 3) return bfail(PIC_ERR_ARG, "each extent must be >= order + 2 and >= 3");
            if (!(B.d[a] > 0.0) || !std::isfinite(B.d[a])) return bfail(PIC_ERR_ARG, "cell sizes must be positive");
            s += 1.0 / (B.d[a] * B.d[a]);
        }
        dt_lim = std::min(dt_lim, 1.0 / std::sqrt(s));
        B.C = int64_t(B.n[0]) * B.n[1] * B.n[2];
        // each box starts on a multiple of 64 cells: the tile kernel's current
        // flush adds float4s at 16-byte aligned addresses of the box's arrays
        B.cbase = C;
        C += (B.C + 63) / 64 * 64;
    }
    if (C >= (int64_t(1) << 31) - 1) return bfail(PIC_ERR_ARG, "total cell count must be below 2^31");
    if (!(dt > 0.0)) {
        if (!(cfl > 0.0) || cfl > 1.0) return bfail(PIC_ERR_ARG, "need dt > 0 or 0 < cfl <= 1");
        dt = cfl * dt_lim;
    }
    if (dt > dt_lim) return bfail(PIC_ERR_CFL, "dt exceeds the Yee Courant limit of a box");
    auto* b = new pic_batch;
    b->box = std::move(boxes);
    pic_ctx& P = b->pool;
    P.dt = dt;
    P.prec = precision;
    P.rsize = precision == PIC_FP64 ? 8 : 4;
    P.stream = static_cast<cudaStream_t>(cuda_stream);
    P.order = 0;
    std::memset(&P.g, 0, sizeof(P.g));
    P.g.C = C;
    for (auto& B : b->box) B.g = box_geom(B, b->tune.tile);
    auto bail = [&](cudaError_t e, const char* what) {
        pic_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? bfail(PIC_ERR_OOM, what) : bcuda(e, what);
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&P.device)) != cudaSuccess) return bail(e, "device");
    if (!P.stream) {  // the legacy default stream cannot be captured into a graph
        if ((e = cudaStreamCreateWithFlags(&P.stream, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(e, "stream");
        b->own_stream = true;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P.device) == cudaSuccess && sms > 0) b->sms = sms;
    char* fb = nullptr;
    if ((e = cudaMalloc(&fb, 9 * size_t(C) * P.rsize)) != cudaSuccess) return bail(e, "field allocation");
    for (int i = 0; i < 9; ++i) P.F[i] = fb + i * size_t(C) * P.rsize;
    if ((e = cudaMemset(fb, 0, 9 * size_t(C) * P.rsize)) != cudaSuccess) return bail(e, "field zeroing");
    if ((e = cudaMalloc(&P.count, size_t(C) * sizeof(int))) != cudaSuccess) return bail(e, "count allocation");
    if ((e = cudaMemset(P.count, 0, size_t(C) * sizeof(int))) != cudaSuccess) return bail(e, "count zeroing");
    if ((e = cudaMalloc(&P.offsets, (size_t(C) + 1) * sizeof(int))) != cudaSuccess) return bail(e, "offsets");
    if ((e = cudaMemset(P.offsets, 0, (size_t(C) + 1) * sizeof(int))) != cudaSuccess) return bail(e, "offsets");
    P.scan_chunks = int(pic::scan_status_words(C) - 1);
    if ((e = cudaMalloc(&P.scan_status, pic::scan_status_words(C) * sizeof(unsigned long long))) != cudaSuccess)
        return bail(e, "scan status");
    if ((e = cudaMalloc(&P.err, 8 * sizeof(unsigned))) != cudaSuccess) return bail(e, "error word");
    if ((e = cudaMemset(P.err, 0, 8 * sizeof(unsigned))) != cudaSuccess) return bail(e, "error word");
    if ((e = cudaMalloc(&P.d_step, sizeof(long long))) != cudaSuccess) return bail(e, "step counter");
    if ((e = cudaMemset(P.d_step, 0, sizeof(long long))) != cudaSuccess) return bail(e, "step counter");
    if ((e = cudaMalloc(&P.dsum, 32 * sizeof(double))) != cudaSuccess) return bail(e, "diagnostics scratch");
    if ((e = cudaMalloc(&P.stage, pic::kStageBytes)) != cudaSuccess) return bail(e, "host-copy staging buffer");
    if ((e = pic::configure_batch_kernels()) != cudaSuccess) return bail(e, "configure batch kernels");
    *out = b;
    return PIC_OK;
}

pic_status pic_batch_destroy(pic_batch* b) {
    if (!b) return PIC_OK;
    pic_ctx& P = b->pool;
    if (P.stream) cudaStreamSynchronize(P.stream);
    else cudaDeviceSynchronize();
    drop_graph(b);
    pic::free_particles(&P);
    cudaFree(P.F[0]);
    cudaFree(P.count);
    cudaFree(P.offsets);
    cudaFree(P.scan_status);
    cudaFree(P.err);
    cudaFree(P.d_step);
    cudaFree(P.dsum);
    cudaFree(P.stage);
    cudaFree(b->tab);
    if (b->own_stream) cudaStreamDestroy(P.stream);
    delete b;
    return PIC_OK;
}

pic_status pic_batch_load_particles(pic_batch* b, double q, double m, const int64_t* counts, const double* x,
                                    const double* y, const double* z, const double* ux, const double* uy,
                                    const double* uz, const double* w, int on_device) {
    if (pic_status s = check_batch(b)) return s;
    if (!counts) return bfail(PIC_ERR_ARG, "NULL counts");
    if (!std::isfinite(q) || !std::isfinite(m) || !(m > 0.0)) return bfail(PIC_ERR_ARG, "q must be finite, m > 0");
    int64_t total = 0;
    for (size_t i = 0; i < b->box.size(); ++i) {
        if (counts[i] < 0) return bfail(PIC_ERR_ARG, "negative particle count");
        total += counts[i];
    }
    if (total >= (int64_t(1) << 31)) return bfail(PIC_ERR_ARG, "total particle count must be below 2^31");
    const double* src[7] = {x, y, z, ux, uy, uz, w};
    if (total > 0)
        for (auto p : src)
            if (!p) return bfail(PIC_ERR_ARG, "particle array is NULL");
    pic_ctx& P = b->pool;
    BCUDA(P.stream ? cudaStreamSynchronize(P.stream) : cudaDeviceSynchronize());
    drop_graph(b);
    b->loaded = false;
    if (total > P.cap || P.cap == 0) {
        pic::free_particles(&P);
        cudaError_t e = pic::alloc_particles(&P, total);
        if (e != cudaSuccess) {
            pic::free_particles(&P);
            return e == cudaErrorMemoryAllocation ? bfail(PIC_ERR_OOM, "particle allocation") : bcuda(e, "alloc");
        }
    }
    P.q = q;
    P.m = m;
    P.np = total;
    P.cur = 0;
    P.step = 0;
    int64_t pb = 0;
    for (size_t i = 0; i < b->box.size(); ++i) {
        b->box[i].pbase = pb;
        b->box[i].np = counts[i];
        pb += counts[i];
    }
    double* staged = nullptr;
    const double* dsrc[7];
    if (total > 0 && !on_device) {
        BCUDA(cudaMalloc(&staged, 7 * size_t(total) * sizeof(double)));
        for (int i = 0; i < 7; ++i) {
            cudaError_t e = cudaMemcpyAsync(staged + i * total, src[i], total * sizeof(double), cudaMemcpyHostToDevice,
                                            P.stream);
            if (e != cudaSuccess) {
                cudaFree(staged);
                return bcuda(e, "particle upload");
            }
            dsrc[i] = staged + i * total;
        }
    } else {
        for (int i = 0; i < 7; ++i) dsrc[i] = src[i];
    }
    pic_status st = PIC_OK;
    BCUDA(cudaMemsetAsync(P.err, 0, 8 * sizeof(unsigned), P.stream));
    for (size_t i = 0; i < b->box.size() && st == PIC_OK; ++i) {
        BoxInfo& B = b->box[i];
        if (B.np == 0) {
            B.w_max = 0.0;
            continue;
        }
        pic_ctx v = make_view(b, int(i));
        v.cur = 0;
        const double* bs[7];
        for (int a = 0; a < 7; ++a) bs[a] = dsrc[a] + B.pbase;
        cudaError_t e = pic::launch_load_particles(&v, bs, B.np);
        unsigned hw[8];
        if (e == cudaSuccess) e = cudaMemcpyAsync(hw, P.err, sizeof(hw), cudaMemcpyDeviceToHost, P.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(P.stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(P.err + 6, 0, 2 * sizeof(unsigned), P.stream);
        if (e != cudaSuccess) {
            st = bcuda(e, "batch particle load");
            break;
        }
        b->launches += 1;
        if (hw[0]) st = bfail(PIC_ERR_ARG, "non-finite particle value");
        unsigned long long bits = (unsigned long long)hw[6] | ((unsigned long long)hw[7] << 32);
        std::memcpy(&B.w_max, &bits, sizeof(double));
    }
    if (staged) {
        cudaStreamSynchronize(P.stream);
        cudaFree(staged);
    }
    if (st != PIC_OK) {
        cudaMemsetAsync(P.err, 0, 8 * sizeof(unsigned), P.stream);
        cudaStreamSynchronize(P.stream);
        P.np = 0;
        return st;
    }
    b->loaded = true;
    if (pic_status s = build_tables(b)) return s;
    BCUDA(batch_sort(b));
    b->launches += 3;
    // the tables hold pointers for both buffer roles; nothing to rebuild after the sort
    return read_error(b);
}

pic_status pic_batch_step(pic_batch* b, int32_t nsteps) {
    if (pic_status s = check_batch(b)) return s;
    if (nsteps < 0) return bfail(PIC_ERR_ARG, "nsteps < 0");
    if (!b->loaded) return bfail(PIC_ERR_STATE, "no particles loaded");
    if (nsteps == 0) return PIC_OK;
    if (pic_status s = ensure_graph(b, nsteps)) return s;
    BCUDA(launch_graph(b));
    return read_error(b);
}

pic_status pic_batch_set_tuning(pic_batch* b, const pic_batch_tuning* t) {
    if (pic_status s = check_batch(b)) return s;
    if (!t || !valid_tuning(*t))
        return bfail(PIC_ERR_ARG, "tuning: tile extents powers of two <= 8, run in [0, 64], sort_every in [1, 64]");
    if (b->loaded) BCUDA(cudaStreamSynchronize(b->pool.stream));
    if (pic_status s = apply_tuning(b, *t, true)) return s;
    return b->loaded ? read_error(b) : PIC_OK;
}

pic_status pic_batch_get_tuning(pic_batch* b, pic_batch_tuning* t) {
    if (pic_status s = check_batch(b)) return s;
    if (!t) return bfail(PIC_ERR_ARG, "NULL output");
    *t = b->tune;
    return PIC_OK;
}

pic_status pic_batch_autotune(pic_batch* b, int32_t trial_steps, pic_batch_tuning* best, double* best_ms) {
    if (pic_status s = check_batch(b)) return s;
    if (!b->loaded) return bfail(PIC_ERR_STATE, "no particles loaded");
    if (trial_steps < 1 || trial_steps > 1000) return bfail(PIC_ERR_ARG, "trial_steps must be in [1, 1000]");
    pic_ctx& P = b->pool;
    BCUDA(cudaStreamSynchronize(P.stream));
    const pic_batch_tuning orig = b->tune;
    pic::StateLayout L(&P);
    pic::DeviceBlock store;
    if (store.alloc(L.total) != cudaSuccess) {
        cudaGetLastError();
        return bfail(PIC_ERR_OOM, "autotune state store");
    }
    pic::StateMeta meta;
    BCUDA(pic::save_state(&P, L, store.p, meta));
    cudaEvent_t ev[2];
    BCUDA(cudaEventCreate(&ev[0]));
    BCUDA(cudaEventCreate(&ev[1]));
    const int tiles[][3] = {{8, 8, 8}, {4, 8, 8}, {4, 4, 8}, {4, 4, 4}};
    const int runs[] = {0, 1, 4};
    const int sorts[] = {1, 2, 4};
    pic_batch_tuning win = orig;
    double win_ms = INFINITY;
    pic_status st = PIC_OK;
    for (const auto& tl : tiles)
        for (int run : runs)
            for (int se : sorts) {
                if (st != PIC_OK) break;
                pic_batch_tuning t{{tl[0], tl[1], tl[2]}, run, se};
                // back to the stored state (keys in the original tile shape), then to t
                cudaError_t e = pic::restore_state(&P, L, store.p, meta);
                if (e != cudaSuccess) {
                    st = bcuda(e, "autotune restore");
                    break;
                }
                if ((st = apply_tuning(b, orig, false)) != PIC_OK) break;
                if ((st = apply_tuning(b, t, true)) != PIC_OK) break;
                // one untimed step, then the timed replay of trial_steps steps
                if ((st = ensure_graph(b, 1)) != PIC_OK) break;
                if ((e = launch_graph(b)) != cudaSuccess) {
                    st = bcuda(e, "autotune warm-up");
                    break;
                }
                if ((st = ensure_graph(b, trial_steps)) != PIC_OK) break;
                cudaEventRecord(ev[0], P.stream);
                if ((e = launch_graph(b)) != cudaSuccess) {
                    st = bcuda(e, "autotune trial");
                    break;
                }
                cudaEventRecord(ev[1], P.stream);
                if ((e = cudaEventSynchronize(ev[1])) != cudaSuccess) {
                    st = bcuda(e, "autotune trial");
                    break;
                }
                if ((st = read_error(b)) != PIC_OK) break;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[0], ev[1]);
                const double per = double(ms) / trial_steps;
                if (per < win_ms) {
                    win_ms = per;
                    win = t;
                }
            }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    // restore the stored state and switch to the winner
    cudaError_t e = pic::restore_state(&P, L, store.p, meta);
    if (e != cudaSuccess) return bcuda(e, "autotune restore");
    if (pic_status s = apply_tuning(b, orig, false)) return s;
    if (st != PIC_OK) return st;
    if (pic_status s = apply_tuning(b, win, true)) return s;
    BCUDA(cudaStreamSynchronize(P.stream));
    if (best) *best = win;
    if (best_ms) *best_ms = win_ms;
    return read_error(b);
}

pic_status pic_batch_get_field(pic_batch* b, int32_t box, int32_t which, double* dst, int on_device) {
    if (pic_status s = check_box(b, box)) return s;
    pic_ctx v = make_view(b, box);
    return pic_get_field(&v, which, dst, on_device);
}

pic_status pic_batch_set_field(pic_batch* b, int32_t box, int32_t which, const double* src, int on_device) {
    if (pic_status s = check_box(b, box)) return s;
    pic_ctx v = make_view(b, box);
    return pic_set_field(&v, which, src, on_device);
}

pic_status pic_batch_get_particles(pic_batch* b, int32_t box, double* x, double* y, double* z, double* ux,
                                   double* uy, double* uz, double* w, int32_t* id, int on_device) {
    if (pic_status s = check_box(b, box)) return s;
    pic_ctx v = make_view(b, box);
    return pic_get_particles(&v, x, y, z, ux, uy, uz, w, id, on_device);
}

pic_status pic_batch_diagnostics(pic_batch* b, int32_t box, double out[4]) {
    if (pic_status s = check_box(b, box)) return s;
    pic_ctx v = make_view(b, box);
    pic_status s = pic_diagnostics(&v, out);
    b->launches += v.launches;
    return s;
}

pic_status pic_batch_info(pic_batch* b, int32_t box, int64_t* num_particles, int64_t* num_cells, int64_t* steps,
                          double* dt) {
    if (pic_status s = check_batch(b)) return s;
    if (box < -1 || box >= int32_t(b->box.size())) return bfail(PIC_ERR_ARG, "box index out of range");
    if (num_particles) *num_particles = box < 0 ? b->pool.np : b->box[size_t(box)].np;
    if (num_cells) *num_cells = box < 0 ? b->pool.g.C : b->box[size_t(box)].C;
    if (steps) *steps = b->pool.step;
    if (dt) *dt = b->pool.dt;
    return PIC_OK;
}

pic_status pic_batch_launch_count(pic_batch* b, int64_t* n) {
    if (pic_status s = check_batch(b)) return s;
    if (!n) return bfail(PIC_ERR_ARG, "NULL output");
    *n = b->launches;
    return PIC_OK;
}

}  // extern "C"
