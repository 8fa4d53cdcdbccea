// C-ABI of libpic: context lifetime, validation, particle loading, the step
// loop (CUDA-graph replay per step kind), getters/setters, diagnostics,
// per-kernel timing.  Declarations and the contract: include/pic.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "pic_ctx.h"

namespace {

thread_local std::string g_last_error;

pic_status fail(pic_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

pic_status cuda_fail(cudaError_t e, const char* where) {
    return fail(PIC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PIC_CUDA(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

}  // namespace

namespace pic {

void free_particles(pic_ctx* c) {
    for (int b = 0; b < 2; ++b) {
        cudaFree(c->P[b].a[0]);
        c->P[b] = pic::PartBuf();
    }
    cudaFree(c->old[0]);
    for (auto& o : c->old) o = nullptr;
    c->oldkey = nullptr;
    c->sortbin = nullptr;
    cudaFree(c->outl);
    c->outl = nullptr;
    cudaFree(c->perm);
    c->perm = nullptr;
    c->tile_perm = false;
    c->np = c->cap = 0;
    c->have_old = false;
}

// The split API's old positions and moves and the old cell keys (also the
// bins of pic_sort_particles), allocated for the particle capacity on first use.
cudaError_t alloc_scratch(pic_ctx* c) {
    if (c->old[0]) return cudaSuccess;
    auto align = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t cap = size_t(c->cap < 1 ? 1 : c->cap);
    const size_t per = align(cap * c->rsize);
    char* ob = nullptr;
    cudaError_t e = cudaMalloc(&ob, 6 * per + align(cap * sizeof(int)));
    if (e != cudaSuccess) return e;
    for (int i = 0; i < 6; ++i) c->old[i] = ob + i * per;
    c->oldkey = reinterpret_cast<int*>(ob + 6 * per);
    c->sortbin = c->oldkey;  // pic_sort_particles ends any split-API step, so the two never overlap
    return cudaSuccess;
}

// One allocation per particle buffer: 7 real arrays, key, id.
cudaError_t alloc_particles(pic_ctx* c, int64_t n) {
    const size_t rs = c->rsize;
    const size_t cap = size_t(n < 1 ? 1 : n);
    auto align = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t per = align(cap * rs);
    const size_t ints = align(cap * sizeof(int));
    for (int b = 0; b < 2; ++b) {
        char* base = nullptr;
        cudaError_t e = cudaMalloc(&base, 7 * per + 2 * ints);
        if (e != cudaSuccess) return e;
        for (int i = 0; i < 7; ++i) c->P[b].a[i] = base + i * per;
        c->P[b].key = reinterpret_cast<int*>(base + 7 * per);
        c->P[b].id = reinterpret_cast<int*>(base + 7 * per + ints);
    }
    cudaError_t e = cudaMalloc(&c->outl, ints);
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&c->perm, ints);
    if (e != cudaSuccess) return e;
    c->cap = int64_t(cap);
    return cudaSuccess;
}

// Larger particle buffers for a moving-window context whose plasma has
// outgrown them (particles that travel with the window stay in the box while
// the front keeps filling): the current buffer's np particles move to buffer
// 0 of the new pair in the same order; the split-API scratch is dropped and
// comes back on first use.
cudaError_t grow_particles(pic_ctx* c, int64_t need) {
    const int64_t cap2 = std::max<int64_t>(need, c->cap + c->cap / 4);
    pic_ctx fresh;
    fresh.rsize = c->rsize;
    cudaError_t e = alloc_particles(&fresh, cap2);
    if (e != cudaSuccess) {
        free_particles(&fresh);
        return e;
    }
    const PartBuf& src = c->P[c->cur];
    const size_t n = size_t(c->np);
    for (int i = 0; i < 7 && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(fresh.P[0].a[i], src.a[i], n * c->rsize, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(fresh.P[0].key, src.key, n * sizeof(int), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(fresh.P[0].id, src.id, n * sizeof(int), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free_particles(&fresh);
        return e;
    }
    const int64_t np = c->np;
    free_particles(c);
    c->P[0] = fresh.P[0];
    c->P[1] = fresh.P[1];
    c->outl = fresh.outl;
    c->cap = fresh.cap;
    c->np = np;
    c->cur = 0;
    c->perm = fresh.perm;
    return cudaSuccess;
}

}  // namespace pic

namespace {

using pic::alloc_particles;
using pic::free_particles;

// ---- kernel launch bookkeeping (counts, optional timing) -------------------
// In timing mode every launch is bracketed by a pair of events from a pool on
// the context stream; the pairs are resolved into per-kernel totals when the
// timings are read.
struct PendingTiming {
    cudaEvent_t a, b;
    int timer;
};
std::vector<PendingTiming>& pending(pic_ctx* c);
cudaEvent_t pool_event(pic_ctx* c);

struct Launch {
    pic_ctx* c;
    int timer = -1;
    cudaEvent_t a = nullptr;
    Launch(pic_ctx* ctx, const char* name) : c(ctx) {
        if (!c->timing) return;
        for (int i = 0; i < c->ntimers; ++i)
            if (std::strcmp(c->timers[i].name, name) == 0) timer = i;
        if (timer < 0 && c->ntimers < 16) {
            timer = c->ntimers++;
            c->timers[timer] = {name, 0.0, 0};
        }
        a = pool_event(c);
        if (a) cudaEventRecord(a, c->stream);
    }
    cudaError_t done(cudaError_t e) {
        if (e != cudaSuccess || !c->timing || !a || timer < 0) return e;
        cudaEvent_t b = pool_event(c);
        if (!b) return e;
        cudaEventRecord(b, c->stream);
        pending(c).push_back({a, b, timer});
        return e;
    }
};

int g_capture_kernels = 0;
bool g_capturing = false;

// Stale errors of earlier, already handled runtime calls would otherwise be
// picked up by the cudaGetLastError() that follows each launch.
cudaError_t clear_stale(const char* where) {
    cudaError_t s = cudaGetLastError();
    if (s != cudaSuccess) {
        g_last_error = std::string("stale CUDA error before ") + where + ": " + cudaGetErrorString(s);
        if (std::getenv("PIC_DEBUG_SYNC")) std::fprintf(stderr, "libpic: %s\n", g_last_error.c_str());
    }
    return s;
}

bool debug_sync() {
    static const bool on = std::getenv("PIC_DEBUG_SYNC") != nullptr;
    return on;
}

// With PIC_DEBUG_SYNC set, every counted launch is followed by a stream
// synchronisation and a failure names the kernel on stderr.
cudaError_t counted(pic_ctx* c, const char* name, int kernels, cudaError_t (*fn)(pic_ctx*)) {
    clear_stale(name);
    Launch l(c, name);
    cudaError_t e = l.done(fn(c));
    if (e == cudaSuccess && debug_sync() && !g_capturing) {
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            g_last_error = std::string("kernel ") + name + ": " + cudaGetErrorString(e);
            std::fprintf(stderr, "libpic: %s\n", g_last_error.c_str());
        }
    }
    if (e == cudaSuccess) {
        if (g_capturing) g_capture_kernels += kernels;
        else c->launches += kernels;
    }
    return e;
}

// The particles' keys changed outside a counting tile step: a histogram the
// count array holds no longer matches them.
void keys_changed(pic_ctx* c) {
    if (c->count_state == 1) c->count_state = 2;
}

// count := the histogram of the sort bins (all zero again first if stale).
cudaError_t run_hist(pic_ctx* c) {
    cudaError_t e;
    if (c->count_state != 0 &&
        (e = cudaMemsetAsync(c->count, 0, (size_t(c->g.C) + 1) * sizeof(int), c->stream)) != cudaSuccess)
        return e;
    return counted(c, "k_hist", 1, pic::launch_hist);
}

// A full sort (every particle array moved); count is zero afterwards.
cudaError_t run_sort(pic_ctx* c) {
    cudaError_t e;
    if ((e = run_hist(c)) != cudaSuccess) return e;
    if ((e = counted(c, "k_scan", 1, pic::launch_scan)) != cudaSuccess) return e;
    if ((e = counted(c, "k_scatter", 1, pic::launch_scatter)) != cudaSuccess) return e;
    c->cur = 1 - c->cur;
    c->count_state = 0;
    return cudaSuccess;
}

// The tile kernel needs the particles in tile order of the current offsets;
// after pic_sort_particles with coarse or random bins they are not.
cudaError_t ensure_tile_order(pic_ctx* c) {
    if (c->sorted || c->np == 0) return cudaSuccess;
    cudaError_t e = run_sort(c);
    if (e != cudaSuccess) return e;
    c->sorted = true;
    c->since_sort = 0;
    return cudaSuccess;
}

cudaError_t yee_b_half(pic_ctx* c) { return pic::launch_yee_b(c, 0.5 * c->dt); }

cudaError_t run_yee(pic_ctx* c) {
    cudaError_t e;
    if ((e = counted(c, "k_yee_b", 1, yee_b_half)) != cudaSuccess) return e;
    if ((e = counted(c, "k_yee_e", 1, pic::launch_yee_e)) != cudaSuccess) return e;
    if ((e = counted(c, "k_yee_b", 1, yee_b_half)) != cudaSuccess) return e;
    return counted(c, "k_step_counter", 1, pic::launch_step_counter);
}

// The particle half and the field half of a step.  With two field sets the
// tile kernel deposits J into the other set and the one-pass Yee update
// writes E and B there from the current set's; the sets then swap roles.
// With one set (CKC) J goes into the current set and the three in-place
// passes follow.
// `count_next`: the tile kernel also counts its particles' new keys into the
// (all-zero) count array, so that the next step's sort needs no histogram.
cudaError_t run_tile_and_fields(pic_ctx* c, bool count_next = false) {
    cudaError_t e;
    if (c->filter_passes > 0 && (e = counted(c, "k_filter_z", 1, pic::launch_filter)) != cudaSuccess) return e;
    c->count_into = count_next && c->count_state == 0;
    c->j_other = c->Fo[0] != nullptr;
    e = counted(c, "k_tile_step", 2, pic::launch_tile_step);
    c->j_other = false;
    if (e != cudaSuccess) c->count_state = 2;  // whatever the launch left in count
    else if (c->count_into) c->count_state = 1;
    else keys_changed(c);
    c->count_into = false;
    if (e != cudaSuccess) return e;
    if (!c->Fo[0]) return run_yee(c);
    if ((e = counted(c, "k_yee_fused", 1, pic::launch_yee_fused)) != cudaSuccess) return e;
    pic::swap_field_sets(c);
    return cudaSuccess;
}

// One full step as queued work.  `with_sort` runs the counting sort first, as
// a permutation: histogram, scan, then the slots as perm; the tile kernel
// moves each particle from the other buffer into its sorted slot of the
// current one while it pushes it (the data moves once a step).
cudaError_t enqueue_step(pic_ctx* c, bool with_sort, bool count_next) {
    cudaError_t e;
    if (with_sort) {
        // the previous step's tile kernel may have counted the keys already
        if (c->count_state != 1 && (e = run_hist(c)) != cudaSuccess) return e;
        if ((e = counted(c, "k_scan", 1, pic::launch_scan)) != cudaSuccess) return e;
        if ((e = counted(c, "k_scatter_perm", 1, pic::launch_scatter_perm)) != cudaSuccess) return e;
        c->count_state = 0;
        c->cur = 1 - c->cur;
        c->tile_perm = c->np > 0;
    }
    e = run_tile_and_fields(c, count_next);
    c->tile_perm = false;
    return e;
}

// Particle count after a sort with open z: the removed ones went to the last bin.
cudaError_t read_live_count(pic_ctx* c) {
    int live = 0;
    cudaError_t e = cudaMemcpyAsync(&live, c->offsets + c->g.C, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) c->np = live;
    return e;
}

cudaError_t window_shift(pic_ctx* c) { return pic::launch_window_shift(c); }
cudaError_t inject(pic_ctx* c) { return pic::launch_inject(c); }

// One step with the moving window.  Unless the particles are sorted and
// compact already (after a load or a call's final sort), the step begins
// with the counting sort as a permutation: the removed particles (last bin)
// are left out of it, the live count is read back (the step's one wait), and
// the tile kernel carries only live particles into the sorted buffer.  Then
// the tile kernel (particles leaving z get the removed key), Yee, and the
// window shifts (fields and particles down one cell, front slab filled with
// plasma) as often as speed * t has passed the next cell.  The particles are
// left unsorted, with the removed ones still in place; finish_window_steps
// sorts and compacts them once at the end of pic_step.
pic_status run_window_step(pic_ctx* c) {
    if (!c->sorted) {
        PIC_CUDA(run_hist(c));
        PIC_CUDA(counted(c, "k_scan", 1, pic::launch_scan));
        PIC_CUDA(counted(c, "k_scatter_perm", 1, pic::launch_scatter_perm));
        c->count_state = 0;
        c->cur = 1 - c->cur;
        PIC_CUDA(read_live_count(c));
        c->tile_perm = c->np > 0;
    }
    const cudaError_t et = run_tile_and_fields(c);
    c->tile_perm = false;
    PIC_CUDA(et);
    c->sorted = false;
    c->step += 1;
    const double t = double(c->step) * c->dt;
    while (c->window_speed > 0.0 && c->window_speed * t >= double(c->shifts + 1) * c->g.d[2]) {
        PIC_CUDA(counted(c, "k_window_shift", c->np > 0 ? 2 : 1, window_shift));
        c->shifts += 1;
        if (c->inj_ppc > 0) {
            const int64_t total = int64_t(c->g.n[0]) * c->g.n[1] * c->inj_ppc;
            if (c->np + total > c->cap) {
                const cudaError_t e = pic::grow_particles(c, c->np + 4 * total);
                if (e == cudaErrorMemoryAllocation) return fail(PIC_ERR_OOM, "particle buffers for the injected plasma");
                PIC_CUDA(e);
            }
            PIC_CUDA(counted(c, "k_inject", 1, inject));
            c->np += total;
            c->next_id += total;
        }
    }
    c->since_sort = 1;
    return PIC_OK;
}

// After a call's window steps: one full sort that also drops the removed
// particles, so that between calls the particles are sorted, compact and
// only live ones.
pic_status finish_window_steps(pic_ctx* c) {
    if (c->sorted) return PIC_OK;
    PIC_CUDA(run_sort(c));
    PIC_CUDA(read_live_count(c));
    c->since_sort = 1;
    c->sorted = true;
    return PIC_OK;
}

// One step of pic_step's direct path: sort at the cadence, tile kernel, Yee.
cudaError_t run_one_step(pic_ctx* c) {
    const bool sort_now = c->since_sort >= c->sort_every;
    const int since_after = sort_now ? 1 : c->since_sort + 1;
    cudaError_t e = enqueue_step(c, sort_now, since_after >= c->sort_every);
    if (e != cudaSuccess) return e;
    if (sort_now) c->since_sort = 0;
    c->since_sort += 1;
    c->step += 1;
    return cudaSuccess;
}

}  // namespace

namespace pic {

cudaError_t save_state(pic_ctx* c, const StateLayout& L, char* dst, StateMeta& m) {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(dst, c->P[c->cur].a[0], L.part, cudaMemcpyDeviceToDevice, c->stream))) return e;
    if ((e = cudaMemcpyAsync(dst + L.part, c->F[0], 9 * size_t(L.C) * L.rs, cudaMemcpyDeviceToDevice, c->stream)))
        return e;
    if ((e = cudaMemcpyAsync(dst + L.part + L.fields, c->offsets, (size_t(L.C) + 1) * sizeof(int),
                             cudaMemcpyDeviceToDevice, c->stream)))
        return e;
    if ((e = cudaMemcpyAsync(dst + L.part + L.fields + L.offs, c->d_step, sizeof(long long),
                             cudaMemcpyDeviceToDevice, c->stream)))
        return e;
    m.cur = c->cur;
    m.since_sort = c->since_sort;
    m.sorted = c->sorted;
    m.step = c->step;
    return cudaSuccess;
}

cudaError_t restore_state(pic_ctx* c, const StateLayout& L, const char* src, const StateMeta& m) {
    cudaError_t e;
    keys_changed(c);
    if ((e = cudaMemcpyAsync(c->P[m.cur].a[0], src, L.part, cudaMemcpyDeviceToDevice, c->stream))) return e;
    if ((e = cudaMemcpyAsync(c->F[0], src + L.part, 9 * size_t(L.C) * L.rs, cudaMemcpyDeviceToDevice, c->stream)))
        return e;
    if ((e = cudaMemcpyAsync(c->offsets, src + L.part + L.fields, (size_t(L.C) + 1) * sizeof(int),
                             cudaMemcpyDeviceToDevice, c->stream)))
        return e;
    if ((e = cudaMemcpyAsync(c->d_step, src + L.part + L.fields + L.offs, sizeof(long long),
                             cudaMemcpyDeviceToDevice, c->stream)))
        return e;
    c->cur = m.cur;
    c->since_sort = m.since_sort;
    c->sorted = m.sorted;
    c->step = m.step;
    return cudaSuccess;
}

}  // namespace pic

namespace {

using pic::DeviceBlock;
using pic::StateLayout;
using pic::StateMeta;
using pic::restore_state;
using pic::save_state;

// Adjoint arrays: lamx, lamu (3 x cap each), lamE, lamB, lamJ (3 x C each),
// lamA (one double), one block.
size_t adj_work_bytes(const pic_ctx* c) {
    const size_t cap = size_t(c->cap < 1 ? 1 : c->cap);
    return 6 * cap * c->rsize + 9 * size_t(c->g.C) * c->rsize + 256;
}

pic::AdjBuffers adj_buffers(const pic_ctx* c, char* base) {
    pic::AdjBuffers b;
    const size_t cap = size_t(c->cap < 1 ? 1 : c->cap);
    const size_t pn = cap * c->rsize, fc = size_t(c->g.C) * c->rsize;
    b.lamA = reinterpret_cast<double*>(base);
    char* p = base + 256;
    for (int a = 0; a < 3; ++a) b.lamx[a] = p + a * pn;
    p += 3 * pn;
    for (int a = 0; a < 3; ++a) b.lamu[a] = p + a * pn;
    p += 3 * pn;
    for (int a = 0; a < 3; ++a) b.lamE[a] = p + a * fc;
    for (int a = 0; a < 3; ++a) b.lamB[a] = p + (3 + a) * fc;
    for (int a = 0; a < 3; ++a) b.lamJ[a] = p + (6 + a) * fc;
    return b;
}

// Work space of pic_step_adjoint: the stored states (checkpoints, one
// segment's per-step states, the final state), the adjoint arrays and the
// staging of dL/du0 for a host destination, each 256-byte aligned.
struct AdjSpace {
    int nseg = 0, nstates = 0;
    size_t states = 0, work = 0, out = 0, total = 0;
    AdjSpace(const pic_ctx* c, int nsteps, int k) {
        auto align = [](size_t b) { return (b + 255) & ~size_t(255); };
        nseg = (nsteps + k - 1) / k;
        const int seg_slots = nsteps > 0 ? (nsteps < k ? nsteps : k) - 1 : 0;
        nstates = nseg + seg_slots + 1;
        states = align(size_t(nstates) * StateLayout(c).total);
        work = align(adj_work_bytes(c));
        out = align(3 * size_t(c->cap < 1 ? 1 : c->cap) * sizeof(double));
        total = states + work + out;
    }
};

template <typename Fn> cudaError_t adj_counted(pic_ctx* c, int kernels, Fn fn) {
    clear_stale("adjoint kernels");
    cudaError_t e = fn();
    if (e == cudaSuccess && debug_sync()) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) c->launches += kernels;
    return e;
}

pic_status read_error_word(pic_ctx* c) {
    unsigned hw[4] = {0, 0, 0, 0};
    PIC_CUDA(cudaMemcpyAsync(hw, c->err, sizeof(hw), cudaMemcpyDeviceToHost, c->stream));
    PIC_CUDA(cudaStreamSynchronize(c->stream));
    const unsigned h = hw[0];
    if (h == 0) return PIC_OK;
    // after a failed step the count array may hold anything: the next sort
    // clears it and counts afresh
    c->count_state = 2;
    PIC_CUDA(cudaMemsetAsync(c->err, 0, sizeof(hw), c->stream));
    PIC_CUDA(cudaStreamSynchronize(c->stream));
    if (h & pic::ERRBIT_CHECK) {
        char buf[160];
        std::snprintf(buf, sizeof(buf), "self-check failed at site %u, value 0x%08x%08x", hw[1], hw[3], hw[2]);
        return fail(PIC_ERR_STATE, buf);
    }
    if (h & pic::ERRBIT_TIMEOUT) return fail(PIC_ERR_TIMEOUT, "a bounded device-side wait ran out");
    if (h & pic::ERRBIT_RANGE) return fail(PIC_ERR_STATE, "a particle cell key was out of range");
    return fail(PIC_ERR_PARTICLE, "a particle became non-finite or moved a cell or more in one step");
}

pic_status check_ctx(pic_ctx* c) {
    if (!c) return fail(PIC_ERR_ARG, "null context");
    return PIC_OK;
}

struct TimingState {
    std::vector<PendingTiming> pend;
    std::vector<cudaEvent_t> free_ev;
    std::vector<cudaEvent_t> all;
};

TimingState& tstate(pic_ctx* c) {
    if (!c->tstate) c->tstate = new TimingState();
    return *static_cast<TimingState*>(c->tstate);
}

std::vector<PendingTiming>& pending(pic_ctx* c) { return tstate(c).pend; }

cudaEvent_t pool_event(pic_ctx* c) {
    TimingState& t = tstate(c);
    if (t.free_ev.empty()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        t.all.push_back(e);
        return e;
    }
    cudaEvent_t e = t.free_ev.back();
    t.free_ev.pop_back();
    return e;
}

// Call after the stream has drained.
void resolve_timings(pic_ctx* c) {
    if (!c->tstate) return;
    TimingState& t = tstate(c);
    for (const PendingTiming& p : t.pend) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess && p.timer < c->ntimers) {
            c->timers[p.timer].ms += ms;
            c->timers[p.timer].launches += 1;
        }
        t.free_ev.push_back(p.a);
        t.free_ev.push_back(p.b);
    }
    t.pend.clear();
}

void destroy_timing(pic_ctx* c) {
    if (!c->tstate) return;
    TimingState& t = tstate(c);
    for (cudaEvent_t e : t.all) cudaEventDestroy(e);
    delete &t;
    c->tstate = nullptr;
}

}  // namespace

namespace pic {
// lets other translation units report through pic_last_error()
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace pic

extern "C" {

const char* pic_last_error(void) { return g_last_error.c_str(); }

pic_status pic_init_grid(const pic_grid_desc* desc, void* cuda_stream, pic_ctx** out) {
    if (!out) return fail(PIC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(PIC_ERR_ARG, "desc is NULL");
    const pic_grid_desc& D = *desc;
    if (D.order < 1 || D.order > 3) return fail(PIC_ERR_ARG, "order must be 1, 2 or 3");
    if (D.precision != PIC_FP64 && D.precision != PIC_FP32_MIXED) return fail(PIC_ERR_ARG, "unknown precision");
    if (D.sort_every < 1) return fail(PIC_ERR_ARG, "sort_every must be >= 1");
    if (D.window_axis != -1 && D.window_axis != 2) return fail(PIC_ERR_ARG, "window_axis must be -1 or 2 (z)");
    if (D.window_axis == 2) {
        if (!(D.window_speed >= 0.0 && D.window_speed <= 1.0))
            return fail(PIC_ERR_ARG, "window_speed must be in [0, 1] (units of c)");
        if (D.sort_every != 1) return fail(PIC_ERR_ARG, "a moving window needs sort_every == 1");
    }
    int64_t C = 1;
    for (int a = 0; a < 3; ++a) {
        if (D.n[a] < D.order + 2 || D.n[a] < 3) return fail(PIC_ERR_ARG, "each extent must be >= order + 2 and >= 3");
        if (!(D.d[a] > 0.0) || !std::isfinite(D.d[a])) return fail(PIC_ERR_ARG, "cell sizes must be finite and > 0");
        C *= D.n[a];
    }
    if (C >= (int64_t(1) << 31) - 1) return fail(PIC_ERR_ARG, "too many cells (limit 2^31 - 2)");
    if (D.solver != 0 && D.solver != 1) return fail(PIC_ERR_ARG, "solver must be 0 (Yee) or 1 (CKC)");
    if (D.solver == 1 && !(D.d[0] == D.d[1] && D.d[1] == D.d[2]))
        return fail(PIC_ERR_ARG, "the CKC solver needs cubic cells");
    const double cfl_dt = D.solver == 1 ? D.d[0]
                                        : 1.0 / std::sqrt(1.0 / (D.d[0] * D.d[0]) + 1.0 / (D.d[1] * D.d[1]) +
                                                          1.0 / (D.d[2] * D.d[2]));
    double dt = D.dt;
    if (dt == 0.0) {
        if (!(D.cfl > 0.0 && D.cfl <= 1.0)) return fail(PIC_ERR_ARG, "cfl must be in (0, 1] when dt == 0");
        dt = D.cfl * cfl_dt;
    }
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(PIC_ERR_ARG, "dt must be finite and > 0");
    if (dt > cfl_dt) return fail(PIC_ERR_CFL, "dt exceeds the Courant limit (Yee 1/sqrt(sum 1/d^2), CKC dx)");

    pic_ctx* c = new pic_ctx();
    c->dt = dt;
    c->prec = D.precision;
    c->order = D.order;
    c->sort_every = D.sort_every;
    c->seed = D.seed;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->rsize = D.precision == PIC_FP64 ? 8 : 4;
    cudaGetDevice(&c->device);
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || c->sms < 1) {
        cudaGetLastError();
        c->sms = 1;
    }
    pic::Geom& g = c->g;
    // Tiles: 4 x 4 x 32 cells when the grid allows (a warp's lanes then walk
    // one z-row of cells), else the largest powers of two up to 8 per axis.
    int T[3];
    const bool given = D.tile[0] > 0 || D.tile[1] > 0 || D.tile[2] > 0;
    if (!given) {
        if (D.n[0] % 4 == 0 && D.n[1] % 4 == 0 && D.n[2] % 32 == 0) {
            T[0] = 4, T[1] = 4, T[2] = 32;
        } else {
            for (int a = 0; a < 3; ++a) {
                T[a] = 8;
                while (T[a] > 1 && D.n[a] % T[a] != 0) T[a] >>= 1;
            }
        }
    } else {
        for (int a = 0; a < 3; ++a) T[a] = D.tile[a];
    }
    for (int a = 0; a < 3; ++a)
        if (!is_pow2(T[a]) || D.n[a] % T[a] != 0) {
            delete c;
            return fail(PIC_ERR_ARG, "tile extents must be powers of two dividing the grid");
        }
    if (T[0] <= 8 && T[1] <= 8 && T[2] <= 8) c->layout = 0;
    else if (T[0] <= 4 && T[1] <= 4 && T[2] <= 32) c->layout = D.precision == PIC_FP32_MIXED && D.order == 1 ? 2 : 1;
    else {
        delete c;
        return fail(PIC_ERR_ARG, "tiles must fit 8x8x8 or 4x4x32 cells");
    }
    for (int a = 0; a < 3; ++a) {
        g.n[a] = D.n[a];
        g.d[a] = D.d[a];
        g.L[a] = D.n[a] * D.d[a];
        g.T[a] = T[a];
        g.lT[a] = ilog2(T[a]);
        g.nt[a] = D.n[a] / T[a];
    }
    g.cpt = g.T[0] * g.T[1] * g.T[2];
    g.C = C;
    g.ntiles = int64_t(g.nt[0]) * g.nt[1] * g.nt[2];
    g.kbase = 0;
    g.zopen = D.window_axis == 2 ? 1 : 0;
    c->window = D.window_axis == 2;
    c->solver = D.solver;
    c->window_speed = c->window ? D.window_speed : 0.0;

    auto bail = [&](cudaError_t e, const char* what) {
        pic_destroy(c);
        return e == cudaErrorMemoryAllocation ? fail(PIC_ERR_OOM, what) : cuda_fail(e, what);
    };
    cudaError_t e;
    // Two field sets with the plain Yee solver (the one-pass update writes the
    // other set), one with CKC (its three in-place passes).
    for (int s = 0; s < (c->solver == 0 ? 2 : 1); ++s) {
        char* fb = nullptr;
        if ((e = cudaMalloc(&fb, 9 * C * c->rsize)) != cudaSuccess) return bail(e, "field allocation");
        c->fblock[s] = fb;
        for (int i = 0; i < 9; ++i) (s == 0 ? c->F : c->Fo)[i] = fb + i * C * c->rsize;
        if ((e = cudaMemset(fb, 0, 9 * C * c->rsize)) != cudaSuccess) return bail(e, "field zeroing");
    }
    if (c->Fo[0] && (e = pic::configure_yee_fused()) != cudaSuccess) return bail(e, "Yee kernel configuration");
    // one bin more than cells (removed particles, open z) and its offset
    if ((e = cudaMalloc(&c->count, (C + 1) * sizeof(int))) != cudaSuccess) return bail(e, "count allocation");
    if ((e = cudaMemset(c->count, 0, (C + 1) * sizeof(int))) != cudaSuccess) return bail(e, "count zeroing");
    if ((e = cudaMalloc(&c->offsets, (C + 2) * sizeof(int))) != cudaSuccess) return bail(e, "offsets allocation");
    if ((e = cudaMemset(c->offsets, 0, (C + 2) * sizeof(int))) != cudaSuccess) return bail(e, "offsets zeroing");
    c->scan_chunks = int(pic::scan_status_words(C + g.zopen) - 1);
    if ((e = cudaMalloc(&c->scan_status, pic::scan_status_words(C + 1) * sizeof(unsigned long long))) != cudaSuccess)
        return bail(e, "scan state allocation");
    if ((e = cudaMalloc(&c->err, 8 * sizeof(unsigned))) != cudaSuccess) return bail(e, "error word allocation");
    if ((e = cudaMemset(c->err, 0, 8 * sizeof(unsigned))) != cudaSuccess) return bail(e, "error word");
    if ((e = pic::configure_tile_kernels(c)) != cudaSuccess) return bail(e, "tile kernel configuration");
    pic::setup_tile_tma(c);
    if ((e = cudaMalloc(&c->d_step, sizeof(long long))) != cudaSuccess) return bail(e, "step counter allocation");
    if ((e = cudaMemset(c->d_step, 0, sizeof(long long))) != cudaSuccess) return bail(e, "step counter");
    if ((e = cudaMalloc(&c->dsum, 32 * sizeof(double))) != cudaSuccess) return bail(e, "diagnostics scratch");
    if ((e = cudaMalloc(&c->stage, pic::kStageBytes)) != cudaSuccess) return bail(e, "host-copy staging buffer");
    *out = c;
    return PIC_OK;
}

pic_status pic_destroy(pic_ctx* c) {
    if (!c) return PIC_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    free_particles(c);
    cudaFree(c->fblock[0]);
    cudaFree(c->fblock[1]);
    cudaFree(c->count);
    cudaFree(c->offsets);
    cudaFree(c->scan_status);
    cudaFree(c->err);
    cudaFree(c->d_step);
    cudaFree(c->dsum);
    cudaFree(c->stage);
    cudaFree(c->adj_space);
    cudaFree(c->rho);
    cudaFree(c->Fg);
    destroy_timing(c);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    delete c;
    return PIC_OK;
}

pic_status pic_load_particles(pic_ctx* c, double q, double m, int64_t n, const double* x, const double* y,
                              const double* z, const double* ux, const double* uy, const double* uz, const double* w,
                              int on_device) {
    if (pic_status s = check_ctx(c)) return s;
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(PIC_ERR_ARG, "particle count must be in [0, 2^31)");
    if (!std::isfinite(q) || !std::isfinite(m) || !(m > 0.0)) return fail(PIC_ERR_ARG, "q must be finite, m > 0");
    const double* src[7] = {x, y, z, ux, uy, uz, w};
    if (n > 0)
        for (auto p : src)
            if (!p) return fail(PIC_ERR_ARG, "particle array is NULL");
    PIC_CUDA(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    // moving window: room for the plasma the window brings in (a full box of
    // it plus two slabs: the removed particles of a step go at the next sort)
    int64_t need = n;
    if (c->window && c->inj_ppc > 0) {
        const int64_t slab = int64_t(c->g.n[0]) * c->g.n[1] * c->inj_ppc;
        need = std::max<int64_t>(n, c->g.C * c->inj_ppc) + 2 * slab;
    }
    if (need > c->cap || c->cap == 0) {
        free_particles(c);
        cudaError_t e = alloc_particles(c, need);
        if (e != cudaSuccess) {
            free_particles(c);
            return e == cudaErrorMemoryAllocation ? fail(PIC_ERR_OOM, "particle allocation") : cuda_fail(e, "alloc");
        }
    }
    c->q = q;
    c->m = m;
    c->np = n;
    c->cur = 0;
    c->have_old = false;
    PIC_CUDA(cudaMemsetAsync(c->err, 0, 8 * sizeof(unsigned), c->stream));
    clear_stale("k_load");
    // Host arrays in pinned (page-locked, mapped) memory are read by the load
    // kernel itself over the host link; other host memory goes through a
    // device staging buffer of at most 2^23 particles, one chunk at a time.
    double* staged = nullptr;
    cudaError_t e = cudaSuccess;
    int64_t loads = 0;
    if (n > 0 && !on_device) {
        const double* mapped[7];
        bool all_mapped = true;
        for (int i = 0; i < 7 && all_mapped; ++i) {
            cudaPointerAttributes at;
            if (cudaPointerGetAttributes(&at, src[i]) != cudaSuccess) {
                cudaGetLastError();
                all_mapped = false;
            } else {
                all_mapped = at.type == cudaMemoryTypeHost && at.devicePointer != nullptr;
                mapped[i] = static_cast<const double*>(at.devicePointer);
            }
        }
        if (all_mapped) {
            e = pic::launch_load_particles(c, mapped, n, 0);
            loads = 1;
        } else {
            // the staging buffer is reused chunk after chunk: stream order keeps
            // each copy behind the load kernel of the chunk before
            const int64_t chunk = std::min<int64_t>(n, int64_t(pic::kStageBytes / (7 * sizeof(double))));
            staged = static_cast<double*>(c->stage);
            for (int64_t b0 = 0; e == cudaSuccess && b0 < n; b0 += chunk) {
                const int64_t cnt = std::min(chunk, n - b0);
                const double* part[7];
                for (int i = 0; i < 7 && e == cudaSuccess; ++i) {
                    e = cudaMemcpyAsync(staged + i * chunk, src[i] + b0, size_t(cnt) * sizeof(double),
                                        cudaMemcpyHostToDevice, c->stream);
                    part[i] = staged + i * chunk;
                }
                if (e == cudaSuccess) e = pic::launch_load_particles(c, part, cnt, b0);
                loads += 1;
            }
        }
    } else {
        e = pic::launch_load_particles(c, src, n, 0);
        loads = n > 0 ? 1 : 0;
    }
    if (e == cudaSuccess) c->launches += loads;
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, n > 0 ? "particle load kernel" : "particle load");
    unsigned hw[8];
    PIC_CUDA(cudaMemcpy(hw, c->err, sizeof(hw), cudaMemcpyDeviceToHost));
    PIC_CUDA(cudaMemset(c->err, 0, sizeof(hw)));
    if (hw[0]) {
        c->np = 0;
        return fail(PIC_ERR_ARG, "non-finite particle value");
    }
    {
        unsigned long long bits = (unsigned long long)hw[6] | ((unsigned long long)hw[7] << 32);
        double wm;
        std::memcpy(&wm, &bits, sizeof(wm));
        c->w_max = n > 0 ? wm : 0.0;
        if (c->window && c->inj_ppc > 0)  // the injected plasma's weight bounds the deposit's fixed-point scale too
            c->w_max = std::max(c->w_max, c->inj_n0 * c->g.d[0] * c->g.d[1] * c->g.d[2] / c->inj_ppc);
    }
    c->next_id = n;
    c->shifts = 0;
    c->step = 0;
    if (c->graph) {  // the deposit scale is a kernel argument baked into the graph
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    e = run_sort(c);
    if (e != cudaSuccess) return cuda_fail(e, "initial sort");
    if (c->window && (e = read_live_count(c)) != cudaSuccess) return cuda_fail(e, "initial sort");
    c->since_sort = 0;
    c->sorted = true;
    return read_error_word(c);
}

pic_status pic_set_window_plasma(pic_ctx* c, int32_t ppc, double n0, double ramp_start, double ramp_length) {
    if (pic_status s = check_ctx(c)) return s;
    if (!c->window) return fail(PIC_ERR_STATE, "the context has no moving window (window_axis = 2)");
    if (c->cap > 0) return fail(PIC_ERR_STATE, "set the injected plasma before pic_load_particles");
    if (ppc < 0 || ppc > 64 || !(n0 >= 0.0) || !std::isfinite(n0) || !std::isfinite(ramp_start) ||
        !(ramp_length >= 0.0) || !std::isfinite(ramp_length))
        return fail(PIC_ERR_ARG, "ppc in [0, 64], finite n0 >= 0, finite ramp_start, finite ramp_length >= 0");
    c->inj_ppc = ppc;
    c->inj_n0 = n0;
    c->inj_ramp_start = ramp_start;
    c->inj_ramp_length = ramp_length;
    return PIC_OK;
}

pic_status pic_set_particle_algorithms(pic_ctx* c, int32_t pusher, int32_t gather) {
    if (pic_status s = check_ctx(c)) return s;
    if (pusher < 0 || pusher > 1 || gather < 0 || gather > 1)
        return fail(PIC_ERR_ARG, "pusher must be 0 (Boris) or 1 (Vay), gather 0 (momentum) or 1 (energy)");
    PIC_CUDA(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    if (c->graph) {  // the choice is a kernel argument baked into the graph
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    c->pusher = pusher;
    c->egather = gather;
    return PIC_OK;
}

pic_status pic_get_window(pic_ctx* c, int64_t* shifts, double* z_lab) {
    if (pic_status s = check_ctx(c)) return s;
    if (shifts) *shifts = c->shifts;
    if (z_lab) *z_lab = double(c->shifts) * c->g.d[2];
    return PIC_OK;
}

pic_status pic_gather_push(pic_ctx* c) {
    if (pic_status s = check_ctx(c)) return s;
    if (c->window) return fail(PIC_ERR_STATE, "the split API runs periodic grids only");
    if (c->np == 0) return fail(PIC_ERR_STATE, "no particles loaded");
    if (cudaError_t e = pic::alloc_scratch(c))
        return e == cudaErrorMemoryAllocation ? fail(PIC_ERR_OOM, "split-API scratch") : cuda_fail(e, "scratch");
    if (c->filter_passes > 0) PIC_CUDA(counted(c, "k_filter_z", 1, pic::launch_filter));
    PIC_CUDA(counted(c, "k_gather_push", 1, pic::launch_gather_push_global));
    keys_changed(c);
    c->have_old = true;
    return PIC_OK;
}

pic_status pic_deposit(pic_ctx* c) {
    if (pic_status s = check_ctx(c)) return s;
    if (c->window) return fail(PIC_ERR_STATE, "the split API runs periodic grids only");
    if (!c->have_old) return fail(PIC_ERR_STATE, "pic_deposit needs a preceding pic_gather_push");
    PIC_CUDA(counted(c, "k_deposit", 1, pic::launch_deposit_global));
    return PIC_OK;
}

pic_status pic_sort_particles(pic_ctx* c, int32_t bin_shift) {
    if (pic_status s = check_ctx(c)) return s;
    if (bin_shift < -1 || bin_shift > 30) return fail(PIC_ERR_ARG, "bin_shift must be in [-1, 30]");
    if (c->window) return fail(PIC_ERR_STATE, "a moving-window context keeps its own sort");
    c->have_old = false;
    if (c->np == 0) return PIC_OK;
    if (bin_shift == 0) {
        PIC_CUDA(run_sort(c));
        c->sorted = true;
        c->since_sort = 0;
        return PIC_OK;
    }
    if (cudaError_t e = pic::alloc_scratch(c))
        return e == cudaErrorMemoryAllocation ? fail(PIC_ERR_OOM, "sort bins") : cuda_fail(e, "scratch");
    c->sort_shift = bin_shift;
    cudaError_t e = counted(c, "k_bin_keys", 1, pic::launch_bin_keys);
    if (e == cudaSuccess) e = run_sort(c);
    c->sort_shift = 0;
    if (bin_shift < 0) c->reorders += 1;
    PIC_CUDA(e);
    c->sorted = false;
    return PIC_OK;
}

pic_status pic_yee_step(pic_ctx* c) {
    if (pic_status s = check_ctx(c)) return s;
    PIC_CUDA(run_yee(c));
    c->step += 1;
    c->since_sort += 1;
    return PIC_OK;
}

pic_status pic_step(pic_ctx* c, int32_t nsteps) {
    if (pic_status s = check_ctx(c)) return s;
    if (nsteps < 0) return fail(PIC_ERR_ARG, "nsteps < 0");
    if (c->np == 0) return fail(PIC_ERR_STATE, "no particles loaded");
    int32_t left = nsteps;
    if (nsteps > 0) PIC_CUDA(ensure_tile_order(c));
    if (c->window) {
        for (; left > 0; --left)
            if (pic_status s = run_window_step(c)) return s;
        if (pic_status s = finish_window_steps(c)) return s;
        c->have_old = false;
        return read_error_word(c);
    }
    // With a sort every step, two consecutive steps return the particle
    // double buffer to its starting role, so a captured pair of steps can be
    // replayed as one graph launch.
    const bool use_graph = c->stream != nullptr && !c->timing && c->sort_every == 1;
    if (use_graph && left >= 2 && c->count_state != 1) {
        // the captured pair of steps takes the histogram from the step before
        PIC_CUDA(run_hist(c));
        c->count_state = 1;
    }
    if (use_graph) {
        while (left >= 2) {
            if (!c->graph || c->graph_cur != c->cur || c->graph_fpar != c->fpar) {
                if (c->graph) {
                    cudaGraphExecDestroy(c->graph);
                    c->graph = nullptr;
                }
                const int cur0 = c->cur, fpar0 = c->fpar;
                PIC_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
                g_capturing = true;
                g_capture_kernels = 0;
                cudaError_t e1 = enqueue_step(c, true, true);
                if (e1 == cudaSuccess) e1 = enqueue_step(c, true, true);
                g_capturing = false;
                cudaGraph_t graph = nullptr;
                cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
                c->cur = cur0;
                if (c->fpar != fpar0) pic::swap_field_sets(c);  // a capture that stopped after one step
                if (e1 != cudaSuccess) {
                    if (graph) cudaGraphDestroy(graph);
                    return cuda_fail(e1, "step capture");
                }
                if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
                cudaError_t e3 = cudaGraphInstantiate(&c->graph, graph, 0);
                cudaGraphDestroy(graph);
                if (e3 != cudaSuccess) return cuda_fail(e3, "graph instantiate");
                c->graph_cur = cur0;
                c->graph_fpar = fpar0;
                c->graph_kernels = g_capture_kernels;
            }
            PIC_CUDA(cudaGraphLaunch(c->graph, c->stream));
            c->launches += c->graph_kernels;
            c->step += 2;
            c->since_sort = 1;
            left -= 2;
        }
    }
    for (; left > 0; --left) PIC_CUDA(run_one_step(c));
    c->have_old = false;
    return read_error_word(c);
}

pic_status pic_step_adjoint(pic_ctx* c, int32_t nsteps, int32_t ckpt_every, double* loss, double* dL_dA,
                            double* dL_du0, int on_device) {
    if (pic_status s = check_ctx(c)) return s;
    if (nsteps < 0 || ckpt_every < 1) return fail(PIC_ERR_ARG, "nsteps must be >= 0 and ckpt_every >= 1");
    if (c->window) return fail(PIC_ERR_STATE, "the adjoint runs periodic grids only");
    if (c->pusher || c->egather || c->solver || c->filter_passes)
        return fail(PIC_ERR_STATE,
                    "the adjoint differentiates Boris, momentum-conserving gather and Yee only (no z filter)");
    if (c->np == 0) return fail(PIC_ERR_STATE, "no particles loaded");
    PIC_CUDA(ensure_tile_order(c));
    PIC_CUDA(cudaStreamSynchronize(c->stream));
    if (pic_status s = read_error_word(c)) return s;
    const int k = ckpt_every;
    const AdjSpace sp(c, nsteps, k);
    const int nseg = sp.nseg;
    const int nstates = sp.nstates;  // checkpoints, segment states, final state
    StateLayout L(c);
    // the space kept by pic_reserve_adjoint when it is large enough, else one
    // allocated for this call
    DeviceBlock own;
    char* space = c->adj_space;
    if (!space || c->adj_space_bytes < sp.total) {
        if (own.alloc(sp.total) != cudaSuccess) {
            clear_stale("adjoint work space");
            return fail(PIC_ERR_OOM, "adjoint work space");
        }
        space = own.p;
    }
    char* const states_p = space;
    char* const work_p = space + sp.states;
    char* const out_p = space + sp.states + sp.work;
    auto state_at = [&](int i) { return states_p + size_t(i) * L.total; };
    std::vector<StateMeta> meta(nstates);
    // forward sweep with checkpoints
    for (int s = 0; s < nsteps; ++s) {
        if (s % k == 0) PIC_CUDA(save_state(c, L, state_at(s / k), meta[s / k]));
        PIC_CUDA(run_one_step(c));
    }
    c->have_old = false;
    if (pic_status s = read_error_word(c)) return s;
    const int fin = nstates - 1;
    PIC_CUDA(save_state(c, L, state_at(fin), meta[fin]));
    double diag[4];
    if (pic_status s = pic_diagnostics(c, diag)) return s;
    if (loss) *loss = diag[0];
    // reverse sweep
    pic::AdjBuffers b = adj_buffers(c, work_p);
    PIC_CUDA(cudaMemsetAsync(work_p, 0, adj_work_bytes(c), c->stream));
    PIC_CUDA(adj_counted(c, 6, [&] { return pic::launch_adj_init(c, b); }));
    std::vector<int> view(k);
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int s0 = seg * k, len = (nsteps - s0 < k ? nsteps - s0 : k);
        PIC_CUDA(restore_state(c, L, state_at(seg), meta[seg]));
        view[0] = seg;
        for (int j = 1; j < len; ++j) {
            PIC_CUDA(run_one_step(c));
            view[j] = nseg + j - 1;
            PIC_CUDA(save_state(c, L, state_at(view[j]), meta[view[j]]));
        }
        for (int j = len - 1; j >= 0; --j) {
            const pic::Snapshot snap = L.view(state_at(view[j]));
            const double t = double(meta[view[j]].step) * c->dt;
            PIC_CUDA(adj_counted(c, 3, [&] { return pic::launch_adj_yee(c, b); }));
            PIC_CUDA(adj_counted(c, 1, [&] { return pic::launch_adj_particles(c, b, snap, t); }));
        }
    }
    if (pic_status s = read_error_word(c)) return s;
    if (dL_dA) PIC_CUDA(cudaMemcpyAsync(dL_dA, b.lamA, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (dL_du0) {
        double* dst = on_device ? dL_du0 : reinterpret_cast<double*>(out_p);
        PIC_CUDA(adj_counted(c, 3, [&] { return pic::launch_adj_output(c, b, dst); }));
        if (!on_device)
            PIC_CUDA(cudaMemcpyAsync(dL_du0, dst, 3 * size_t(c->np) * sizeof(double), cudaMemcpyDeviceToHost,
                                     c->stream));
        PIC_CUDA(cudaStreamSynchronize(c->stream));
    }
    PIC_CUDA(restore_state(c, L, state_at(fin), meta[fin]));
    PIC_CUDA(cudaStreamSynchronize(c->stream));
    return read_error_word(c);
}

pic_status pic_reserve_adjoint(pic_ctx* c, int32_t nsteps, int32_t ckpt_every) {
    if (pic_status s = check_ctx(c)) return s;
    if (nsteps < 0 || ckpt_every < 1) return fail(PIC_ERR_ARG, "nsteps must be >= 0 and ckpt_every >= 1");
    PIC_CUDA(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    if (c->adj_space) {
        PIC_CUDA(cudaFree(c->adj_space));
        c->adj_space = nullptr;
        c->adj_space_bytes = 0;
    }
    if (nsteps == 0) return PIC_OK;
    if (c->cap == 0) return fail(PIC_ERR_STATE, "load the particles first (the space is sized by their capacity)");
    const AdjSpace sp(c, nsteps, ckpt_every);
    char* p = nullptr;
    if (cudaMalloc(&p, sp.total) != cudaSuccess) {
        clear_stale("adjoint reservation");
        return fail(PIC_ERR_OOM, "adjoint work space");
    }
    c->adj_space = p;
    c->adj_space_bytes = sp.total;
    return PIC_OK;
}

pic_status pic_get_field(pic_ctx* c, int32_t which, double* dst, int on_device) {
    if (pic_status s = check_ctx(c)) return s;
    if (!c->stage) return fail(PIC_ERR_STATE, "context has no staging buffer");
    if (which < 0 || which > 8 || !dst) return fail(PIC_ERR_ARG, "bad field index or NULL destination");
    const int64_t C = c->g.C;
    clear_stale("field read");
    if (on_device) {
        PIC_CUDA(pic::launch_field_to_f64(c, which, dst, 0, C));
        PIC_CUDA(cudaStreamSynchronize(c->stream));
        return PIC_OK;
    }
    if (c->prec == PIC_FP64) {
        PIC_CUDA(cudaMemcpyAsync(dst, c->F[which], C * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        PIC_CUDA(cudaStreamSynchronize(c->stream));
        return PIC_OK;
    }
    // FP32 values converted on the device, chunk by chunk through the staging buffer
    const int64_t chunk = int64_t(pic::kStageBytes / sizeof(double));
    double* st = static_cast<double*>(c->stage);
    for (int64_t i0 = 0; i0 < C; i0 += chunk) {
        const int64_t cnt = std::min(chunk, C - i0);
        PIC_CUDA(pic::launch_field_to_f64(c, which, st, i0, cnt));
        PIC_CUDA(cudaMemcpyAsync(dst + i0, st, size_t(cnt) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        PIC_CUDA(cudaStreamSynchronize(c->stream));
    }
    return PIC_OK;
}

pic_status pic_set_field(pic_ctx* c, int32_t which, const double* src, int on_device) {
    if (pic_status s = check_ctx(c)) return s;
    if (!c->stage) return fail(PIC_ERR_STATE, "context has no staging buffer");
    if (which < 0 || which > 8 || !src) return fail(PIC_ERR_ARG, "bad field index or NULL source");
    const int64_t C = c->g.C;
    clear_stale("field write");
    if (on_device) {
        PIC_CUDA(pic::launch_field_from_f64(c, which, src, 0, C));
        PIC_CUDA(cudaStreamSynchronize(c->stream));
        return PIC_OK;
    }
    if (c->prec == PIC_FP64) {
        PIC_CUDA(cudaMemcpyAsync(c->F[which], src, C * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        PIC_CUDA(cudaStreamSynchronize(c->stream));
        return PIC_OK;
    }
    const int64_t chunk = int64_t(pic::kStageBytes / sizeof(double));
    double* st = static_cast<double*>(c->stage);
    for (int64_t i0 = 0; i0 < C; i0 += chunk) {
        const int64_t cnt = std::min(chunk, C - i0);
        PIC_CUDA(cudaMemcpyAsync(st, src + i0, size_t(cnt) * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        PIC_CUDA(pic::launch_field_from_f64(c, which, st, i0, cnt));
        PIC_CUDA(cudaStreamSynchronize(c->stream));
    }
    return PIC_OK;
}

pic_status pic_num_particles(pic_ctx* c, int64_t* n) {
    if (pic_status s = check_ctx(c)) return s;
    if (!n) return fail(PIC_ERR_ARG, "NULL output");
    *n = c->np;
    return PIC_OK;
}

pic_status pic_get_particles(pic_ctx* c, double* x, double* y, double* z, double* ux, double* uy, double* uz,
                             double* w, int32_t* id, int on_device) {
    if (pic_status s = check_ctx(c)) return s;
    if (!c->stage) return fail(PIC_ERR_STATE, "context has no staging buffer");
    double* dst[7] = {x, y, z, ux, uy, uz, w};
    if (c->np == 0) return PIC_OK;
    clear_stale("particle read");
    if (on_device) {
        PIC_CUDA(pic::launch_get_particles(c, dst, id, 0, c->np));
        PIC_CUDA(cudaStreamSynchronize(c->stream));
        return PIC_OK;
    }
    // chunk by chunk through the staging buffer: 7 FP64 arrays and the ids of
    // `chunk` particles (64 bytes a particle)
    const int64_t n = c->np;
    const int64_t chunk = int64_t(pic::kStageBytes / 64);
    char* st = static_cast<char*>(c->stage);
    double* sdst[7];
    for (int i = 0; i < 7; ++i) sdst[i] = dst[i] ? reinterpret_cast<double*>(st) + i * chunk : nullptr;
    int32_t* sid = id ? reinterpret_cast<int32_t*>(st + 7 * chunk * sizeof(double)) : nullptr;
    for (int64_t p0 = 0; p0 < n; p0 += chunk) {
        const int64_t cnt = std::min(chunk, n - p0);
        PIC_CUDA(pic::launch_get_particles(c, sdst, sid, p0, cnt));
        for (int i = 0; i < 7; ++i)
            if (dst[i])
                PIC_CUDA(cudaMemcpyAsync(dst[i] + p0, sdst[i], size_t(cnt) * sizeof(double), cudaMemcpyDeviceToHost,
                                         c->stream));
        if (id)
            PIC_CUDA(cudaMemcpyAsync(id + p0, sid, size_t(cnt) * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        PIC_CUDA(cudaStreamSynchronize(c->stream));
    }
    return PIC_OK;
}

pic_status pic_set_external_drive(pic_ctx* c, double amp, double k) {
    if (pic_status s = check_ctx(c)) return s;
    if (!std::isfinite(amp) || !std::isfinite(k)) return fail(PIC_ERR_ARG, "drive parameters must be finite");
    c->drive_amp = amp;
    c->drive_k = k;
    if (c->graph) {  // kernel arguments are baked into the graph
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return PIC_OK;
}

pic_status pic_get_time(pic_ctx* c, int64_t* steps, double* t) {
    if (pic_status s = check_ctx(c)) return s;
    if (steps) *steps = c->step;
    if (t) *t = double(c->step) * c->dt;
    return PIC_OK;
}

pic_status pic_diagnostics(pic_ctx* c, double out[4]) {
    if (pic_status s = check_ctx(c)) return s;
    if (!out) return fail(PIC_ERR_ARG, "NULL output");
    PIC_CUDA(cudaMemsetAsync(c->dsum, 0, 8 * sizeof(double), c->stream));
    clear_stale("diagnostics");
    PIC_CUDA(pic::launch_diagnostics(c, c->dsum));
    c->launches += c->np > 0 ? 3 : 2;
    double h[4];
    PIC_CUDA(cudaMemcpyAsync(h, c->dsum, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    PIC_CUDA(cudaStreamSynchronize(c->stream));
    const double dV = c->g.d[0] * c->g.d[1] * c->g.d[2];
    out[0] = h[0] * dV;
    out[1] = h[1];
    out[2] = h[2];
    unsigned long long bits;
    std::memcpy(&bits, &h[3], sizeof(bits));
    double mx;
    std::memcpy(&mx, &bits, sizeof(mx));
    out[3] = mx;
    return read_error_word(c);
}

// The two FP64 density arrays of the charge and continuity diagnostics,
// allocated on first use.
static pic_status ensure_rho(pic_ctx* c) {
    if (c->rho) return PIC_OK;
    if (cudaMalloc(&c->rho, 2 * size_t(c->g.C) * sizeof(double)) != cudaSuccess) {
        c->rho = nullptr;
        clear_stale("charge density");
        return fail(PIC_ERR_OOM, "charge density arrays");
    }
    c->have_mark = false;
    return PIC_OK;
}

static double* rho_array(pic_ctx* c, int which) { return c->rho + size_t(which) * size_t(c->g.C); }

pic_status pic_charge_density(pic_ctx* c, double* dst, int on_device) {
    if (pic_status s = check_ctx(c)) return s;
    if (!dst) return fail(PIC_ERR_ARG, "NULL destination");
    if (pic_status s = ensure_rho(c)) return s;
    clear_stale("charge density");
    double* r = rho_array(c, 1 - c->rho_mark);  // the marked density stays
    PIC_CUDA(pic::launch_charge_density(c, r));
    c->launches += c->np > 0 ? 1 : 0;
    PIC_CUDA(cudaMemcpyAsync(dst, r, size_t(c->g.C) * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    PIC_CUDA(cudaStreamSynchronize(c->stream));
    return read_error_word(c);
}

pic_status pic_continuity_mark(pic_ctx* c) {
    if (pic_status s = check_ctx(c)) return s;
    if (pic_status s = ensure_rho(c)) return s;
    clear_stale("continuity mark");
    PIC_CUDA(pic::launch_charge_density(c, rho_array(c, c->rho_mark)));
    c->launches += c->np > 0 ? 1 : 0;
    PIC_CUDA(cudaStreamSynchronize(c->stream));
    c->have_mark = true;
    c->mark_step = c->step;
    c->mark_shifts = c->shifts;
    return read_error_word(c);
}

pic_status pic_continuity_residual(pic_ctx* c, double out[3]) {
    if (pic_status s = check_ctx(c)) return s;
    if (!out) return fail(PIC_ERR_ARG, "NULL output");
    if (!c->rho || !c->have_mark) return fail(PIC_ERR_STATE, "no pic_continuity_mark before the step");
    if (c->step != c->mark_step + 1 || c->shifts != c->mark_shifts)
        return fail(PIC_ERR_STATE, "the residual needs exactly one step since the mark and no window shift");
    clear_stale("continuity residual");
    const int m = c->rho_mark;
    PIC_CUDA(pic::launch_charge_density(c, rho_array(c, 1 - m)));
    unsigned long long* d = reinterpret_cast<unsigned long long*>(c->dsum + 16);
    PIC_CUDA(pic::launch_continuity(c, rho_array(c, m), rho_array(c, 1 - m), d));
    c->launches += c->np > 0 ? 2 : 1;
    unsigned long long h[2];
    PIC_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    PIC_CUDA(cudaStreamSynchronize(c->stream));
    double mr, m0;
    std::memcpy(&mr, &h[0], sizeof(double));
    std::memcpy(&m0, &h[1], sizeof(double));
    out[0] = m0 > 0.0 ? mr / m0 : mr;
    out[1] = mr;
    out[2] = m0;
    // the new density is the mark of the next step
    c->rho_mark = 1 - m;
    c->mark_step = c->step;
    c->mark_shifts = c->shifts;
    return read_error_word(c);
}

pic_status pic_set_gather_filter(pic_ctx* c, int32_t passes) {
    if (pic_status s = check_ctx(c)) return s;
    if (passes < 0 || passes > 16) return fail(PIC_ERR_ARG, "passes must be in [0, 16]");
    if (passes > 0 && pic::filter_smem_bytes(c) > 200 * 1024)
        return fail(PIC_ERR_ARG, "the z filter holds a z column in shared memory: nz too large");
    PIC_CUDA(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    if (passes > 0 && !c->Fg) {
        if (cudaMalloc(&c->Fg, 6 * size_t(c->g.C) * c->rsize) != cudaSuccess) {
            c->Fg = nullptr;
            clear_stale("filter allocation");
            return fail(PIC_ERR_OOM, "filtered field copy");
        }
        c->tma_g = pic::encode_eb_tensor_map(&c->tmap_g, c->Fg, c->g.n, c->g.C, c->layout, c->prec);
        PIC_CUDA(pic::configure_filter(c));
    }
    if (c->graph) {  // the gathered arrays are kernel arguments baked into the graph
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    c->filter_passes = passes;
    return PIC_OK;
}

pic_status pic_set_fp64_gamma(pic_ctx* c, double gamma) {
    if (pic_status s = check_ctx(c)) return s;
    if (!(gamma >= 1.0)) return fail(PIC_ERR_ARG, "gamma must be >= 1 (or +infinity)");
    PIC_CUDA(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    if (c->graph) {  // a kernel argument baked into the graph
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    c->gamma_fp64 = gamma;
    return PIC_OK;
}

pic_status pic_sync(pic_ctx* c) {
    if (pic_status s = check_ctx(c)) return s;
    return read_error_word(c);
}

pic_status pic_set_timing(pic_ctx* c, int32_t on) {
    if (pic_status s = check_ctx(c)) return s;
    PIC_CUDA(cudaStreamSynchronize(c->stream));
    resolve_timings(c);
    c->timing = on != 0;
    c->ntimers = 0;
    return PIC_OK;
}

pic_status pic_get_timing(pic_ctx* c, int32_t cap, const char** names, double* ms, int64_t* launches,
                          int32_t* count) {
    if (pic_status s = check_ctx(c)) return s;
    PIC_CUDA(cudaStreamSynchronize(c->stream));
    resolve_timings(c);
    for (int i = 0; i < c->ntimers && i < cap; ++i) {
        if (names) names[i] = c->timers[i].name;
        if (ms) ms[i] = c->timers[i].ms;
        if (launches) launches[i] = c->timers[i].launches;
    }
    if (count) *count = c->ntimers;
    return PIC_OK;
}

pic_status pic_launch_count(pic_ctx* c, int64_t* n) {
    if (pic_status s = check_ctx(c)) return s;
    if (!n) return fail(PIC_ERR_ARG, "NULL output");
    *n = c->launches;
    return PIC_OK;
}

}  // extern "C"
