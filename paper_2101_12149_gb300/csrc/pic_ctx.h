// Host-side context of libpic and the launchers shared between its
// translation units.  Not part of the public C-ABI (see include/pic.h).
#pragma once
#include <cuda.h>  // CUtensorMap (the type only: the encoder is reached through the runtime)
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "pic.h"

namespace pic {

// Error bits of the device error word.
enum : unsigned {
    ERRBIT_PARTICLE = 1u,  // non-finite particle or a move of >= 1 cell
    ERRBIT_TIMEOUT = 2u,   // a bounded wait ran out
    ERRBIT_RANGE = 4u,     // a sort key outside [0, C)
    ERRBIT_CHECK = 8u,     // a device-side self-check failed (see check word); most run in checking builds only
};

// Checking builds (-DPIC_CHECK) verify indices before memory accesses; the
// first failure stores {site, value} in err[1], err[2] and the access is
// skipped.  The error word allocation holds 4 words.

// Particle storage (structure of arrays).  FP64: a[0..6] = x,y,z,ux,uy,uz,w
// (double), key = tile-major cell key.  FP32-mixed: key = tile-major cell key
// (the integer part of the position), a[0..6] = ox,oy,oz (in-cell offsets in
// [0,1)), ux,uy,uz, w (float).  id = load index.
struct PartBuf {
    void* a[7] = {nullptr};
    int* key = nullptr;
    int* id = nullptr;
};

// Grid geometry shared by all kernels.
struct Geom {
    int n[3];      // cells per axis
    int T[3];      // cells per tile per axis (powers of two)
    int lT[3];     // log2 T
    int nt[3];     // tiles per axis
    int cpt;       // cells per tile
    int64_t C;     // cells
    int64_t ntiles;
    double d[3];
    double L[3];
    int kbase;     // added to every cell key (a box's first key in a batch of boxes; 0 otherwise)
    int zopen;     // 1: z is open (moving window): no field beyond the z ends, particles leaving z die
};

// Key of a removed particle: one past the last cell; the sort puts these last.
__host__ __device__ inline int dead_key(const Geom& g) { return g.kbase + int(g.C); }

struct Timer {
    const char* name;
    double ms;
    int64_t launches;
};

}  // namespace pic

struct pic_ctx {
    pic::Geom g;
    double dt = 0.0;
    int prec = PIC_FP64;
    int order = 1;
    int sort_every = 1;
    cudaStream_t stream = nullptr;
    int device = 0;
    size_t rsize = 8;  // bytes per real (8 FP64, 4 FP32-mixed)

    void* F[9] = {nullptr};  // Ex Ey Ez Bx By Bz Jx Jy Jz (the current set)
    // The other set of the same nine arrays (plain Yee solver): a step's
    // current is deposited into it and the one-pass field update writes the
    // new E and B into it, then the two sets swap roles.  Both sets are one
    // allocation each (fblock); fpar says which block is current.
    void* Fo[9] = {nullptr};
    void* fblock[2] = {nullptr, nullptr};
    int fpar = 0;
    bool j_other = false;  // the tile kernel deposits into Fo's J

    int64_t np = 0, cap = 0;
    double q = 0.0, m = 1.0;
    double w_max = 0.0;  // largest |weight| loaded (fixed-point scale of the FP32-mixed deposit)
    pic::PartBuf P[2];
    int cur = 0;
    void* old[6] = {nullptr};  // split API: old position (3 arrays: FP64 x,y,z / FP32-mixed offsets) and move (3),
                               // allocated on first use (alloc_scratch)
    int* oldkey = nullptr;     // FP32-mixed: key of the old position
    bool have_old = false;

    int* outl = nullptr;     // outsider list of the tile kernel [cap]
    int* perm = nullptr;     // the step's sort order [cap] (k_scatter_perm)
    bool tile_perm = false;  // the next tile kernel reads the other buffer through perm
    int layout = 0;          // shared-memory layout of the tile kernel: 0 = up to 8x8x8, 1 = 4x4x32,
                             // 2 = 4x4x32 with a halo of 1 (FP32-mixed, order 1)
    int sms = 1;             // streaming multiprocessors of the device (persistent grids)
    // TMA descriptor of E and B (four dimensions z, y, x, component) whose box
    // is one tile's staged E/B block
    CUtensorMap tmap_eb;
    bool tma = false;
    CUtensorMap tmap_eb_o;  // the other set's E/B
    bool tma_o = false;

    int* count = nullptr;    // per-cell particle counts [C]
    // What count holds: 0 all zero (a scatter leaves it so), 1 the histogram
    // of the current keys (a tile kernel counted its particles' new keys),
    // 2 stale (non-zero, not the current keys: cleared before the next
    // histogram).  count_into: the next tile-kernel launch counts.
    int count_state = 0;
    bool count_into = false;
    int* offsets = nullptr;  // exclusive scan of count [C+1]; tile t owns [offsets[t*cpt], offsets[(t+1)*cpt])
    unsigned long long* scan_status = nullptr;  // look-back words + ticket
    int scan_chunks = 0;
    bool sorted = false;       // particles are in tile order of the current offsets
    int since_sort = 0;
    // sort bins: 0 = cells (the step's sort); > 0 = runs of 2^sort_shift
    // consecutive tile-major cells; -1 = pseudo-random bins (pic_sort_particles)
    int sort_shift = 0;
    int* sortbin = nullptr;    // bin of each particle when sort_shift != 0 [cap]
    uint64_t seed = 0;
    int64_t reorders = 0;      // pic_sort_particles calls with random bins so far

    unsigned* err = nullptr;       // device error word [4] + outsider count [1] + tile queue counter [1]
                                   // (8 words allocated; words 6, 7 carry the load's largest weight)
    long long* d_step = nullptr;   // device copy of the step counter (drive time)
    double* dsum = nullptr;        // diagnostics scratch
    int64_t step = 0;
    double drive_amp = 0.0, drive_k = 0.0;
    int solver = 0;   // 0 Yee, 1 CKC (B update with the transverse-averaged curl)
    int pusher = 0;   // 0 Boris, 1 Vay
    int egather = 0;  // 0 momentum-conserving, 1 energy-conserving gather
    double gamma_fp64 = 1e3;  // FP32-mixed: gamma above which the push's rotation runs in FP64 (inf: never)
    // z filter of the gathered fields: passes (0 = off), the filtered E and B
    // (6 arrays of C values, allocated when first switched on) and their TMA
    // descriptor for the tile kernel
    int filter_passes = 0;
    void* Fg = nullptr;
    CUtensorMap tmap_g;
    bool tma_g = false;

    // charge density and continuity diagnostics: two FP64 density arrays
    // (allocated on first use), the one holding the mark, and the step count
    // and window shifts at the mark
    double* rho = nullptr;
    int rho_mark = 0;
    bool have_mark = false;
    int64_t mark_step = 0, mark_shifts = 0;

    bool timing = false;
    pic::Timer timers[16];
    int ntimers = 0;
    void* tstate = nullptr;  // pending event pairs and the event pool

    // moving window along z (window_axis = 2): speed in units of c, shifts so
    // far, the plasma injected into each new front slab, next particle id
    bool window = false;
    double window_speed = 0.0;
    int64_t shifts = 0;
    int inj_ppc = 0;
    double inj_n0 = 0.0, inj_ramp_start = 0.0, inj_ramp_length = 0.0;
    int64_t next_id = 0;

    cudaGraphExec_t graph = nullptr;
    int graph_cur = 0;
    int graph_fpar = 0;
    int graph_kernels = 0;
    int64_t launches = 0;

    // staging buffer of the host getters and setters (kStageBytes, allocated
    // by pic_init_grid): FP32 fields and particle state pass through it in
    // chunks, converted to or from FP64 on the device
    void* stage = nullptr;
    // adjoint work space kept by pic_reserve_adjoint (null: none)
    char* adj_space = nullptr;
    size_t adj_space_bytes = 0;
};

namespace pic {
constexpr size_t kStageBytes = size_t(32) << 20;
}

namespace pic {

// launchers (pic_kernels.cu)
cudaError_t launch_zero_fields(pic_ctx* c, int first, int count);
cudaError_t launch_tile_step(pic_ctx* c);        // fused gather+push+deposit, tile kernel
cudaError_t configure_tile_kernels(pic_ctx* c);
// encodes c->tmap_eb where the tile kernel can stage by TMA (sets c->tma)
void setup_tile_tma(pic_ctx* c);
// TMA descriptor of the E/B arrays of one box (E and B at `base`, components
// comp_stride values apart, precision `prec`) for tile layout `layout` (0:
// 8x8x8, 1: 4x4x32); false (and a zeroed map) where TMA cannot be used
bool encode_eb_tensor_map(CUtensorMap* map, const void* base, const int n[3], int64_t comp_stride, int layout,
                          int prec);
cudaError_t launch_gather_push_global(pic_ctx* c);
cudaError_t launch_deposit_global(pic_ctx* c);
cudaError_t launch_yee_b(pic_ctx* c, double h);
cudaError_t launch_yee_e(pic_ctx* c);
// One-pass field update from the current set (E, B) and the other set's J
// into the other set's E, B, and the step counter advanced (plain Yee, the
// other set allocated); the caller then swaps the sets (swap_field_sets).
cudaError_t launch_yee_fused(pic_ctx* c);
cudaError_t configure_yee_fused();
void swap_field_sets(pic_ctx* c);

cudaError_t launch_step_counter(pic_ctx* c);
// particles [base, base + n) from arrays that start at particle base
cudaError_t launch_load_particles(pic_ctx* c, const double* const src[7], int64_t n, int64_t base = 0);
// particles [p0, p0 + cnt) (current order) into element 0.. of dst / id
cudaError_t launch_get_particles(pic_ctx* c, double* const dst[7], int32_t* id, int64_t p0, int64_t cnt);
// field values [i0, i0 + cnt) to / from FP64 (dst / src hold cnt values)
cudaError_t launch_field_to_f64(pic_ctx* c, int which, double* dst, int64_t i0, int64_t cnt);
cudaError_t launch_field_from_f64(pic_ctx* c, int which, const double* src, int64_t i0, int64_t cnt);
cudaError_t launch_diagnostics(pic_ctx* c, double* d_out);
// z filter of E, B into c->Fg (pic_set_gather_filter); nothing when off
cudaError_t launch_filter(pic_ctx* c);
cudaError_t configure_filter(const pic_ctx* c);
size_t filter_smem_bytes(const pic_ctx* c);
// nodal charge density of the current particles into rho (C doubles, zeroed first)
cudaError_t launch_charge_density(pic_ctx* c, double* rho);
// out[0] = max |rho1 - rho0 + dt div J| (J: the context's current), out[1] =
// max |rho0| over the nodes the residual covers, as FP64 bit patterns (zeroed first)
cudaError_t launch_continuity(pic_ctx* c, const double* rho0, const double* rho1, unsigned long long* out);
// moving window: move fields and particles down one cell along z (particles
// below z = 0 die), then fill the front slab with plasma at slots [np, np + nx*ny*ppc)
cudaError_t launch_window_shift(pic_ctx* c);
cudaError_t launch_inject(pic_ctx* c);
// bins of pic_sort_particles (sort_shift != 0) into sortbin (pic_sort.cu)
cudaError_t launch_bin_keys(pic_ctx* c);

// adjoint (pic_adjoint.cu)
// Work buffers of the reverse sweep: adjoints of positions (cell units) and
// momenta indexed by particle id, of E, B and J per cell, and of the drive
// amplitude (FP64 accumulator).
struct AdjBuffers {
    void* lamx[3] = {nullptr, nullptr, nullptr};
    void* lamu[3] = {nullptr, nullptr, nullptr};
    void* lamE[3] = {nullptr, nullptr, nullptr};
    void* lamB[3] = {nullptr, nullptr, nullptr};
    void* lamJ[3] = {nullptr, nullptr, nullptr};
    double* lamA = nullptr;
};
// A stored state: one particle buffer (same layout as PartBuf) and the nine
// field arrays, as they were at the start of a step.
struct Snapshot {
    void* a[7] = {nullptr};
    int* key = nullptr;
    int* id = nullptr;
    const void* F[9] = {nullptr};
};
// ---- stored states (adjoint checkpoints, autotuner trials) -------------------
// A device allocation freed on scope exit.
struct DeviceBlock {
    char* p = nullptr;
    cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes < 256 ? 256 : bytes); }
    ~DeviceBlock() {
        if (p) cudaFree(p);
    }
};

// Host-side part of a stored state.
struct StateMeta {
    int cur = 0, since_sort = 0;
    bool sorted = false;
    int64_t step = 0;
};

// Byte layout of one stored state: the current particle buffer (as laid out
// by alloc_particles), the nine field arrays, the cell offsets of the last
// sort and the device step counter.
struct StateLayout {
    size_t per, ints, part, fields, offs, total;
    int64_t C;
    size_t rs;
    explicit StateLayout(const pic_ctx* c) {
        auto align = [](size_t b) { return (b + 255) & ~size_t(255); };
        rs = c->rsize;
        C = c->g.C;
        const size_t cap = size_t(c->cap < 1 ? 1 : c->cap);
        per = align(cap * rs);
        ints = align(cap * sizeof(int));
        part = 7 * per + 2 * ints;
        fields = align(9 * size_t(C) * rs);
        offs = align((size_t(C) + 1) * sizeof(int));
        total = part + fields + offs + 256;
    }
    pic::Snapshot view(char* base) const {
        pic::Snapshot s;
        for (int i = 0; i < 7; ++i) s.a[i] = base + i * per;
        s.key = reinterpret_cast<int*>(base + 7 * per);
        s.id = reinterpret_cast<int*>(base + 7 * per + ints);
        for (int i = 0; i < 9; ++i) s.F[i] = base + part + i * size_t(C) * rs;
        return s;
    }
};

cudaError_t save_state(pic_ctx* c, const StateLayout& L, char* dst, StateMeta& m);
cudaError_t restore_state(pic_ctx* c, const StateLayout& L, const char* src, const StateMeta& m);

// particle buffers (pic_api.cu): one allocation per buffer, 7 real arrays, key, id
cudaError_t alloc_particles(pic_ctx* c, int64_t n);
cudaError_t alloc_scratch(pic_ctx* c);
void free_particles(pic_ctx* c);

cudaError_t launch_adj_init(pic_ctx* c, const AdjBuffers& b);
cudaError_t launch_adj_yee(pic_ctx* c, const AdjBuffers& b);
cudaError_t launch_adj_particles(pic_ctx* c, const AdjBuffers& b, const Snapshot& s, double t);
cudaError_t launch_adj_output(pic_ctx* c, const AdjBuffers& b, double* d_out);

// batch of boxes (pic_batch.cu host side, kernels in pic_kernels.cu)
// One launch of the persistent batch tile kernel over the boxes of one shape
// order, followed by its outsider kernel.
struct BatchTileLaunch {
    int order = 1;
    const void* boxes = nullptr;     // StepArgs<R>[nboxes] (R = double for FP64, float for FP32-mixed)
    const int2* items = nullptr;     // (box, tile) work items, heaviest first
    int nitems = 0;
    int* queue = nullptr;            // work counter, zeroed before the launch
    const int64_t* pbase = nullptr;  // first particle of each box, nboxes + 1 entries
    int nboxes = 0;
    const int* outn = nullptr;       // outsider count and list of this order's boxes
    const int* outl = nullptr;
    int grid = 0;                    // persistent CTAs
};
cudaError_t launch_tile_step_batch(int prec, const BatchTileLaunch& L, cudaStream_t s);
// Yee update of all boxes: yb / ye are YeeArgs<R>[nboxes] with h = dt/2 and
// h = dt; blocks maps each 256-thread block to (box, first cell, cells).
cudaError_t launch_yee_batch(int prec, const void* yb, const void* ye, const int4* blocks, int nblocks,
                             long long* step, cudaStream_t s);
// New cell keys of n particles after a change of tile shape (from -> to).
cudaError_t launch_rekey(int* key, int64_t n, const Geom& from, const Geom& to, cudaStream_t s);
cudaError_t configure_batch_kernels();

// sort (pic_sort.cu)
cudaError_t launch_hist(pic_ctx* c);
cudaError_t launch_scan(pic_ctx* c);
cudaError_t launch_scatter(pic_ctx* c);
// the step's sort as a permutation (perm), the particle data left in place
cudaError_t launch_scatter_perm(pic_ctx* c);
size_t scan_status_words(int64_t C);

}  // namespace pic
