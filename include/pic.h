/*
 * libpic: GB300-native (sm_103a) electromagnetic particle-in-cell hot path.
 *
 * One species of macro-particles on a 3-D periodic Yee grid, advanced by the
 * PIC loop whose GPU port the paper describes (Myers et al., "Porting WarpX
 * to GPU-accelerated platforms", 2021):
 *   field gather with order-p B-spline shapes, p = 1..3 (Sec. 4.1.1 runs
 *     3rd order; fused with the push, Sec. 3.1),
 *   relativistic Boris push and position advance,
 *   Esirkepov charge-conserving current deposition (Sec. 3.4.1),
 *   Yee FDTD update of E and B (Sec. 2.4, Sec. 4.1.1),
 *   per-step counting sort of the particles by cell (Sec. 3.4.2).
 *
 * Conventions.  Normalised units c = eps0 = mu0 = 1.  Node (i,j,k) sits at
 * (i dx, j dy, k dz); the box is periodic with length n*d per axis.  Field
 * arrays are nx*ny*nz values, element (i*ny + j)*nz + k (k fastest) holding
 * the component at its staggered location just above node (i,j,k):
 *   Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2)
 *   Bx(i,j+1/2,k+1/2) By(i+1/2,j,k+1/2) Bz(i+1/2,j+1/2,k)   J like E.
 * Particle momentum is u = gamma v (units of m c); u lives at half steps.
 * One step: gather E^n, B^n at x^n -> Boris u^{n-1/2} -> u^{n+1/2} ->
 * x^{n+1} = x^n + dt u/gamma -> Esirkepov J^{n+1/2} -> B half step, E full
 * step with -dt J, B half step.
 *
 * Ownership.  The context owns every device buffer; they are allocated by
 * pic_init_grid (fields, with the Yee solver in two sets, sort state, a
 * 32 MiB host-copy staging buffer) and
 * pic_load_particles (particle buffers), by the first call that needs an
 * optional one (the split API's scratch, the charge density of
 * pic_charge_density), and by pic_reserve_adjoint; none inside pic_step.
 * Arrays passed in are copied; the caller keeps ownership.  Getters copy out
 * into caller memory.  `on_device` = 1 means the pointer is device memory of
 * the context's GPU, 0 means host memory (pageable or pinned).
 *
 * Errors.  Every call returns a pic_status; nothing throws across the ABI.
 * pic_last_error() gives a message for the calling thread's last failure.
 * Kernels report asynchronous faults (non-finite particle, particle moving a
 * cell or more per step, a scan wait that ran out) in a device error word that
 * pic_step and pic_sync check.
 *
 * Streams.  All work is queued on the stream given to pic_init_grid
 * (NULL = the legacy default stream).  Calls return once the work is queued,
 * except getters to host memory, pic_sync and pic_diagnostics, which wait.
 */
#ifndef LIBPIC_PIC_H
#define LIBPIC_PIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_ctx pic_ctx;

typedef enum {
    PIC_OK = 0,
    PIC_ERR_ARG = 1,      /* invalid argument (NULL, bad order, extents, sizes) */
    PIC_ERR_CFL = 2,      /* dt above the Yee Courant limit 1/sqrt(sum 1/d^2) */
    PIC_ERR_OOM = 3,      /* device allocation failed */
    PIC_ERR_CUDA = 4,     /* a CUDA runtime call failed */
    PIC_ERR_STATE = 5,    /* call out of order (e.g. stepping with no particles) */
    PIC_ERR_PARTICLE = 6, /* a particle became non-finite or moved >= 1 cell in a step */
    PIC_ERR_TIMEOUT = 7   /* a bounded device-side wait ran out */
} pic_status;

enum { PIC_FP64 = 0, PIC_FP32_MIXED = 1 };

enum { PIC_EX = 0, PIC_EY, PIC_EZ, PIC_BX, PIC_BY, PIC_BZ, PIC_JX, PIC_JY, PIC_JZ };

/* Grid and method description (the problem statement of the paper's
 * uniform-plasma runs, Sec. 4.1.1: extents, cell size, dt at a stated
 * Courant number, shape order). */
typedef struct {
    int32_t n[3];        /* cells per axis, each >= order + 2 */
    double d[3];         /* cell size per axis, > 0 */
    double dt;           /* time step; 0 selects dt = cfl / sqrt(sum 1/d^2) */
    double cfl;          /* Courant number used when dt == 0, in (0, 1] */
    int32_t precision;   /* PIC_FP64 or PIC_FP32_MIXED */
    int32_t order;       /* shape order 1..3 */
    int32_t sort_every;  /* counting sort every this many steps (>= 1) */
    int32_t window_axis; /* -1: periodic box; 2: moving window along z (Sec. 4.2): z open (no field
                            beyond the z ends, current there dropped, particles leaving z removed),
                            x, y periodic; needs sort_every = 1 */
    double window_speed; /* window speed in units of c, in [0, 1] (window_axis = 2) */
    uint64_t seed;       /* reserved for generators that run inside the library */
    int32_t tile[3];     /* cells per tile per axis (powers of two dividing n); 0 = automatic */
    int32_t solver;      /* field solver: 0 Yee; 1 CKC (Sec. 4.2: the B update takes each
                            difference of curl E averaged over the two transverse directions
                            with weights (1/4, 1/2, 1/4) per direction; cubic cells only;
                            stable up to dt = dx, so the Courant limit is dx) */
} pic_grid_desc;

/* Create a context: validates the description (PIC_ERR_ARG, PIC_ERR_CFL),
 * allocates the nine field arrays (zeroed) on the current CUDA device and
 * binds `cuda_stream` (a cudaStream_t, may be NULL).  With the Yee solver a
 * second set of nine arrays is allocated too: pic_step writes each step's
 * new E and B (and deposits its J) into the other set, and the two sets then
 * swap roles; getters and setters always address the current set.  *out
 * receives the context; on failure *out is NULL. */
pic_status pic_init_grid(const pic_grid_desc* desc, void* cuda_stream, pic_ctx** out);

/* Load one species: charge q and mass m per unit weight, n particles with
 * positions x,y,z (inside [0, n*d) per axis; values outside are wrapped),
 * momenta ux,uy,uz = gamma v at t = -dt/2, weights w (FP64 arrays of n).
 * Replaces any previous particles, allocates the particle buffers for n,
 * assigns ids 0..n-1 in input order and sorts the particles by cell.
 * on_device = 0: host arrays; when all seven are in pinned (page-locked,
 * device-mapped) memory the load kernel reads them directly over the host
 * link, otherwise they pass through the context's 32 MiB staging buffer
 * (599,186 particles at a time).  Returns when the load is complete.
 * PIC_ERR_ARG if n < 0 or n >= 2^31, a pointer is NULL with n > 0, or a
 * value is non-finite. */
pic_status pic_load_particles(pic_ctx* ctx, double q, double m, int64_t n,
                              const double* x, const double* y, const double* z,
                              const double* ux, const double* uy, const double* uz,
                              const double* w, int on_device);

/* Gather E,B at the particles, Boris push and position advance (one
 * particle per thread, fields read from global memory).  Saves the old
 * positions for pic_deposit.  Does not sort.  Periodic grids only
 * (PIC_ERR_STATE with a moving window), as is pic_deposit. */
pic_status pic_gather_push(pic_ctx* ctx);

/* Zero J and deposit the Esirkepov current of the move made by the last
 * pic_gather_push (one particle per thread, global atomics).
 * PIC_ERR_STATE if no pic_gather_push preceded it. */
pic_status pic_deposit(pic_ctx* ctx);

/* Yee update with the current J: B half step, E full step, B half step. */
pic_status pic_yee_step(pic_ctx* ctx);

/* Reorder the particles now with the counting sort (Sec. 3.4.2 bins the
 * particles by cell and reorders their data; the paper sweeps the bin size
 * and the sort interval).  bin_shift = 0: by cell, in tile-major cell order
 * (the order pic_step keeps); bin_shift in 1..30: by bins of 2^bin_shift
 * consecutive tile-major cells, in no set order within a bin;
 * PIC_ORDER_RANDOM (-1): a pseudo-random order (bins drawn from the particle
 * id, pic_grid_desc.seed and a per-context call counter; the paper has no
 * such call: it stands for the state of a long run without sorting).  With
 * the split API the caller chooses the bins and the cadence.  After anything
 * but a cell sort, the next pic_step or pic_step_adjoint first sorts by cell.
 * Physics is unchanged (results up to the order of floating-point additions);
 * a pic_gather_push not yet followed by pic_deposit is dropped.
 * PIC_ERR_ARG if bin_shift is outside [-1, 30]; PIC_ERR_STATE for a
 * moving-window context. */
enum { PIC_ORDER_RANDOM = -1 };
pic_status pic_sort_particles(pic_ctx* ctx, int32_t bin_shift);

/* nsteps full PIC steps: counting sort (at the sort cadence), fused tile
 * kernel (gather + push + advance + Esirkepov into shared memory, one flush
 * per tile), Yee update.  Checks the device error word at the end.
 * With a moving window (Sec. 4.2: the domain moves with the beam at c, new
 * plasma enters at the front, particles leaving at the back are removed),
 * each step is: a sort that leaves out the particles removed by the step
 * before (the step waits for the live particle count), tile kernel, Yee
 * update, then as often as window_speed * t_{n+1} has reached the next cell
 * the window shift (all fields move down one cell along z with a zero front
 * slab, particles move by -dz and those below z = 0 are removed) and the
 * injection of the front slab's plasma (pic_set_window_plasma).  The call
 * ends with one more sort, so that between calls the particles are sorted
 * and only live ones remain. */
pic_status pic_step(pic_ctx* ctx, int32_t nsteps);

/* Plasma injected into each new front slab of a moving-window context:
 * in every cell of the slab, ppc particles m = 0..ppc-1 at in-cell offset
 * (m + 1/2)/ppc on every axis, at rest, of weight n(z) dV / ppc where the
 * density at lab-frame z (window z + shifts * dz) is 0 below ramp_start,
 * rises linearly over ramp_length (0 = a step) and is n0 beyond; none where
 * it is zero.  Injected particles take ids counting on from the loaded ones,
 * (i ny + j) ppc + m within a slab.  Call before pic_load_particles (it sizes
 * the particle buffers for a full box of this plasma plus two slabs; a step
 * whose injection would exceed them first grows them by a quarter, keeping
 * the particles, or returns PIC_ERR_OOM).  PIC_ERR_STATE without a window. */
pic_status pic_set_window_plasma(pic_ctx* ctx, int32_t ppc, double n0, double ramp_start,
                                 double ramp_length);

/* Particle algorithms (Sec. 4.2 lists both options for the plasma-
 * acceleration run): pusher 0 = Boris (default), 1 = Vay (Vay 2008: the
 * average velocity (v^{n-1/2} + v^{n+1/2})/2 in the magnetic force, which
 * keeps the E x B drift exact at relativistic speed); gather 0 =
 * momentum-conserving (order p along every axis, default), 1 =
 * energy-conserving (order p - 1 along each axis where the component is
 * staggered, the order of the Esirkepov current along its own direction).
 * Applies to pic_step and the split API; pic_step_adjoint needs the defaults
 * (PIC_ERR_STATE otherwise).  PIC_ERR_ARG for other values.  Waits. */
pic_status pic_set_particle_algorithms(pic_ctx* ctx, int32_t pusher, int32_t gather);

/* Number of window shifts so far and the lab-frame z of the window's
 * lower end (shifts * dz).  Either pointer may be NULL. */
pic_status pic_get_window(pic_ctx* ctx, int64_t* shifts, double* z_lab);

/* Discrete adjoint of nsteps PIC steps (the paper has no adjoint; this is
 * the reverse-mode derivative of exactly the step pic_step runs: gather,
 * Boris push, advance, Esirkepov deposit, Yee update).
 *
 * Loss: L = 1/2 sum over cells (|E|^2 + |B|^2) dV after the nsteps steps.
 * Runs the steps forward from the current state, storing the full state
 * (particles and fields) every ckpt_every steps; then, segment by segment from
 * the last, recomputes the segment's per-step states from its checkpoint and
 * runs the reverse kernels: transposed Yee update, then per particle the
 * adjoints of the deposit, advance, Boris rotation, drive and gather.  Cell
 * indices are held fixed (floor has zero derivative).
 *
 * loss: host double, written (may be NULL).
 * dL_dA: host double, written: dL/d(drive amplitude) (may be NULL).
 * dL_du0: 3*n doubles, written (may be NULL): dL/du at the current state,
 *   component-major (all ux, then uy, then uz), each component in particle
 *   load order (by id).  Host memory unless on_device = 1.
 * ckpt_every >= 1.  Work space: about (ceil(nsteps/ckpt_every) + ckpt_every
 *   + 1) stored states plus the adjoint arrays and the staging of dL_du0.
 *   It is the space kept by pic_reserve_adjoint when that is large enough
 *   (then the call allocates nothing); otherwise the call allocates it and
 *   frees it before returning; PIC_ERR_OOM if that fails.
 * On return the context holds the state after the nsteps steps, as after
 * pic_step(ctx, nsteps).  Waits.  PIC_ERR_STATE if no particles are loaded
 * or the context has a moving window (periodic grids only). */
pic_status pic_step_adjoint(pic_ctx* ctx, int32_t nsteps, int32_t ckpt_every, double* loss,
                            double* dL_dA, double* dL_du0, int on_device);

/* Allocate and keep the work space of pic_step_adjoint for nsteps steps
 * with checkpoints every ckpt_every steps at the current particle capacity,
 * so that those adjoint calls (and any shorter ones) allocate nothing inside
 * the step loop.  Replaces an earlier reservation; nsteps = 0 releases it.
 * The space is sized by the particle buffers: a later pic_load_particles
 * with more particles needs a new reservation (until then the adjoint
 * allocates for the call).  PIC_ERR_STATE before pic_load_particles,
 * PIC_ERR_OOM if the allocation fails.  Waits.  (The paper has no adjoint;
 * this follows its Sec. 3.2: device allocation is costly, so buffers are
 * taken once and kept, not allocated inside the time step.) */
pic_status pic_reserve_adjoint(pic_ctx* ctx, int32_t nsteps, int32_t ckpt_every);

/* Copy one field component (PIC_EX..PIC_JZ) out as FP64 / in from FP64.
 * With host memory and the FP32-mixed precision the values pass through the
 * context's 32 MiB staging buffer (converted on the device), chunk by chunk;
 * nothing is allocated.  Waits. */
pic_status pic_get_field(pic_ctx* ctx, int32_t which, double* dst, int on_device);
pic_status pic_set_field(pic_ctx* ctx, int32_t which, const double* src, int on_device);

/* Number of particles held. */
pic_status pic_num_particles(pic_ctx* ctx, int64_t* n);

/* Copy particle state out as FP64 (positions in [0, L)), in the library's
 * current (cell-sorted) order; `id` gives each particle's load index.  Any
 * pointer may be NULL to skip that array.  To host memory the values pass
 * through the context's 32 MiB staging buffer, 524,288 particles at a time;
 * nothing is allocated.  Waits. */
pic_status pic_get_particles(pic_ctx* ctx, double* x, double* y, double* z,
                             double* ux, double* uy, double* uz, double* w,
                             int32_t* id, int on_device);

/* External drive added to the gathered E at each particle (not to the grid):
 * E_y += amp * cos(k x - k t_n), t_n = n dt the time of the gather.  amp = 0
 * switches it off. */
pic_status pic_set_external_drive(pic_ctx* ctx, double amp, double k);

/* Simulation time step count and time (t = steps * dt). */
pic_status pic_get_time(pic_ctx* ctx, int64_t* steps, double* t);

/* Diagnostics (FP64 reductions on the device): out[0] = field energy
 * 1/2 sum(|E|^2+|B|^2) dV, out[1] = kinetic energy sum w m (gamma - 1),
 * out[2] = sum of charge q w, out[3] = max |div B| dV^(1/3).  Waits. */
pic_status pic_diagnostics(pic_ctx* ctx, double out[4]);

/* Nodal charge density of the current particles (Sec. 3.4.1 deposits
 * charge and current; rho sits on the nodes):
 *   rho(i,j,k) = sum_p (q w_p / dV) s_p(x_p/dx - i) s_p(y_p/dy - j) s_p(z_p/dz - k)
 * with the order-p shapes, folded periodically (z open: nodes beyond the z
 * ends take nothing).  Deposited on the device in FP64 whatever the
 * precision (FP32-mixed positions are exact in FP64), order of the additions
 * free.  dst: C doubles, element (i ny + j) nz + k, host or device memory per
 * on_device.  The first call of this or the two continuity calls allocates
 * the diagnostics' two density arrays (2 C doubles), kept until pic_destroy.
 * Waits. */
pic_status pic_charge_density(pic_ctx* ctx, double* dst, int on_device);

/* Discrete continuity of the last step (Sec. 3.4.1: the Esirkepov current
 * conserves charge exactly, rho^{n+1} - rho^n + dt div J^{n+1/2} = 0 node by
 * node).  pic_continuity_mark deposits rho^n of the current particles and
 * keeps it.  After exactly one step (pic_step(ctx, 1), or the split API's
 * gather/push, deposit and Yee calls), pic_continuity_residual deposits
 * rho^{n+1}, forms r = rho^{n+1} - rho^n + dt div J at every node with the
 * step's own current (the context's J arrays; div J the nodal difference of
 * the edge-centred J, periodic) and returns out[0] = max|r| / max|rho^n|,
 * out[1] = max|r|, out[2] = max|rho^n|; rho^{n+1} then becomes the mark, so
 * the two calls chain step by step.  With a moving window the residual
 * covers the z-planes at least order + 2 cells from the z ends (current
 * beyond the ends is dropped and particles leaving are removed) and a window
 * shift since the mark is PIC_ERR_STATE, as is a missing mark or any other
 * number of steps since it.  Waits. */
pic_status pic_continuity_mark(pic_ctx* ctx);
pic_status pic_continuity_residual(pic_ctx* ctx, double out[3]);

/* Filter along z of the fields the particles gather (Sec. 4.2 applies the
 * Godfrey filter to E and B before gathering them; the paper gives no
 * coefficients, so this is the compensated binomial form of that filter
 * family): before each step's gather, E and B are copied through `passes`
 * passes of the stencil (1/4, 1/2, 1/4) along z and one compensation pass
 * (-passes/4, 1 + passes/2, -passes/4), each reading the previous pass's
 * output, periodic along z or zero beyond the z ends with a moving window.
 * The transfer function on a mode e^{ikz} is cos^(2 passes)(k dz/2)
 * (1 + passes sin^2(k dz/2)): long waves pass (1 - O(k^4)), the Nyquist mode
 * is removed.  The particles gather from the filtered copy; the field update
 * advances the unfiltered fields.  passes = 0 switches it off.  The first
 * call with passes > 0 allocates the copy (6 C values).  PIC_ERR_ARG for
 * passes outside [0, 16] or nz beyond the shared-memory column (about 25,600
 * FP32 / 12,800 FP64 cells); pic_step_adjoint needs it off.  Waits. */
pic_status pic_set_gather_filter(pic_ctx* ctx, int32_t passes);

/* FP32-mixed precision: the Lorentz factor above which the push's magnetic
 * rotation (Boris: gamma^- and the rotation; Vay: the solve, for |u'| above
 * it) is computed in FP64 instead of FP32.  Default 1e3; +infinity never
 * switches, 1 always does.  The FP64 path ignores it.  PIC_ERR_ARG for
 * gamma < 1 or NaN.  Waits.  (The paper runs FP64 throughout; Sec. 3.1
 * names reduced precision as a way to cut the memory footprint.) */
pic_status pic_set_fp64_gamma(pic_ctx* ctx, double gamma);

/* Wait for queued work; returns the device error word's status. */
pic_status pic_sync(pic_ctx* ctx);

/* Per-kernel timing: when on, pic_step launches its kernels directly (no
 * graph) between CUDA events on the context stream and accumulates their
 * durations.  pic_get_timing fills up to `cap` entries: kernel name
 * (pointer to a static string), total milliseconds and launch count, and
 * returns the number of kernel kinds in *count.  Waits. */
pic_status pic_set_timing(pic_ctx* ctx, int32_t on);
pic_status pic_get_timing(pic_ctx* ctx, int32_t cap, const char** names, double* ms,
                          int64_t* launches, int32_t* count);

/* Number of kernels this context has launched (graph replays counted per
 * kernel node). */
pic_status pic_launch_count(pic_ctx* ctx, int64_t* n);

/* Counting sort of caller-owned keys that allocates nothing.
 *
 * The paper has no counterpart.  This entry point is for callers that are
 * not allowed to allocate device memory: a host application that gives a
 * library only the buffers it may touch and keeps the device's memory budget
 * to itself, or a loop with timing guarantees where the implicit device-wide
 * synchronisation of cudaMalloc/cudaFree cannot be afforded.  It runs the same
 * histogram and single-pass scan as the particle sort of pic_step, then a
 * scatter of a permutation, on caller arrays.  Its scratch (per-bin counts,
 * the scan's look-back words, an error word) is one static device array of
 * about 16 MiB that every GPU loading the library holds until the process
 * exits; no call allocates or frees anything.
 *
 * keys: n int32 bin indices in [0, nbins) (device memory).
 * offsets: nbins+1 int32 (device, written): offsets[b] is the first slot of
 *   bin b, offsets[nbins] = n (exclusive prefix sum of the histogram).
 * perm: n int32 (device, written): perm[slot] = index of the key placed
 *   there; bin b holds slots [offsets[b], offsets[b+1]), in no set order.
 * nbins: 1 .. 4,194,304 (the scratch limit); larger values give PIC_ERR_ARG.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 *
 * Set-up: the first call on a device (and the first after that device's
 * context was reset) looks up the scratch array's device address with
 * cudaGetSymbolAddress, with that device current; make that first call before
 * any stream capture.  Each call clears the part of the scratch it uses (the
 * array keeps the previous call's contents), then waits for its work to
 * finish and reads the error word.  All calls share the one array, so calls
 * that overlap on the GPU (from other threads or streams) race: serialise
 * them.  A CUDA error already pending on the calling thread is left in place
 * and returned as PIC_ERR_CUDA before anything is launched.
 * PIC_ERR_ARG: bad sizes, NULL arrays, or a key outside [0, nbins) (the
 * offsets then count only the keys inside); PIC_ERR_TIMEOUT: a bounded
 * device-side wait ran out. */
pic_status pic_sort_keys_noalloc(const int32_t* keys, int64_t n, int32_t nbins, int32_t* offsets,
                                 int32_t* perm, void* cuda_stream);

/* ---- batch of independent boxes -----------------------------------------
 *
 * Many independent periodic plasma boxes of uneven sizes (each its own
 * extents, cell size, shape order, particles and fields; one dt for all)
 * stepped together: each step runs one persistent tile kernel per shape
 * order over the (box, tile) work items of all boxes, and pic_batch_step
 * replays its whole step loop as one CUDA graph.  Each box computes exactly
 * what a single-box context with the same extents computes (Sec. 3.1 gather
 * and push, Sec. 3.4.1 Esirkepov deposit, Sec. 2.4 Yee update, Sec. 3.4.2
 * sort); the paper runs one box per GPU and has no batching. */
typedef struct pic_batch pic_batch;

/* Performance knobs (results are unchanged up to the order of floating-point
 * additions): largest tile extent per axis (powers of two <= 8; each box
 * uses the largest power of two not above it that divides its extent),
 * particles per lane run in the tile kernel (0 = automatic: each warp
 * splits its own group of the tile's cells when the particles are spread
 * evenly over the groups, else runs of about one cell's worth),
 * sort cadence in steps (>= 1; between sorts particles that left their tile
 * take a slower global-memory path).  Default {8,8,8}, 0, 1. */
typedef struct {
    int32_t tile[3];
    int32_t run;
    int32_t sort_every;
} pic_batch_tuning;

/* nboxes boxes: n = 3*nboxes extents (each >= order + 2 and >= 3), d =
 * 3*nboxes cell sizes or NULL for unit cells, order = nboxes shape orders
 * (1..3).  dt > 0 is used as given (PIC_ERR_CFL if above any box's Courant
 * limit); dt = 0 takes cfl times the smallest limit.  precision PIC_FP64 or
 * PIC_FP32_MIXED.  Fields start at zero.  Host pointers; all are copied.
 * cuda_stream NULL: the batch creates and owns a non-blocking stream (the
 * legacy default stream cannot be captured into a graph); device inputs
 * must then be complete before the call that reads them. */
pic_status pic_batch_init(int32_t nboxes, const int32_t* n, const double* d, const int32_t* order,
                          double dt, double cfl, int32_t precision, void* cuda_stream,
                          pic_batch** out);

/* Particles of all boxes, one species (q, m): counts[i] particles for box i,
 * the arrays holding box 0's particles first, then box 1's, ...; positions
 * in each box's own coordinates.  Replaces any earlier particles, resets the
 * step count, sorts.  on_device as for pic_load_particles.  Waits. */
pic_status pic_batch_load_particles(pic_batch* b, double q, double m, const int64_t* counts,
                                    const double* x, const double* y, const double* z,
                                    const double* ux, const double* uy, const double* uz,
                                    const double* w, int on_device);

/* nsteps steps of every box (captured once as a CUDA graph per step count
 * and state, then replayed).  Waits and checks the device error word. */
pic_status pic_batch_step(pic_batch* b, int32_t nsteps);

/* Per-box access, as pic_get_field / pic_set_field / pic_get_particles /
 * pic_diagnostics (particle ids are load indices within the box; fields may
 * be set after pic_batch_load_particles). */
pic_status pic_batch_get_field(pic_batch* b, int32_t box, int32_t which, double* dst, int on_device);
pic_status pic_batch_set_field(pic_batch* b, int32_t box, int32_t which, const double* src, int on_device);
pic_status pic_batch_get_particles(pic_batch* b, int32_t box, double* x, double* y, double* z,
                                   double* ux, double* uy, double* uz, double* w, int32_t* id,
                                   int on_device);
pic_status pic_batch_diagnostics(pic_batch* b, int32_t box, double out[4]);

/* Particle and cell counts of one box (box = -1: all boxes), steps taken and
 * dt.  Any output may be NULL. */
pic_status pic_batch_info(pic_batch* b, int32_t box, int64_t* num_particles, int64_t* num_cells,
                          int64_t* steps, double* dt);

/* Switch the knobs (re-keys and re-sorts the particles).  Waits. */
pic_status pic_batch_set_tuning(pic_batch* b, const pic_batch_tuning* t);
pic_status pic_batch_get_tuning(pic_batch* b, pic_batch_tuning* t);

/* Autotuner: from the current state, times trial_steps steps (after one
 * untimed step) of every candidate (tile extents {8,8,8}, {4,8,8}, {4,4,8},
 * {4,4,4} x run {0,1,4} x sort cadence {1,2,4}), restores the state after
 * each, and keeps the fastest; returns it and its milliseconds per step.
 * The simulation state afterwards is the state before the call (re-sorted).
 * Allocates one stored state for the duration of the call.  Waits. */
pic_status pic_batch_autotune(pic_batch* b, int32_t trial_steps, pic_batch_tuning* best,
                              double* best_ms);

/* Number of kernels the batch has launched (graph replays counted per node). */
pic_status pic_batch_launch_count(pic_batch* b, int64_t* n);

/* Release the batch (NULL is allowed). */
pic_status pic_batch_destroy(pic_batch* b);

/* Release every buffer of the context (NULL is allowed). */
pic_status pic_destroy(pic_ctx* ctx);

/* Measured fused multiply-add throughput of the current device in TFLOP/s
 * (FMA = 2 flops): precision PIC_FP32_MIXED times FP32 FMAs, PIC_FP64 FP64
 * FMAs.  Independent register FMA chains on every SM, timed with CUDA events
 * (best of three launches after a warm-up).  The ALU ceiling of the roofline
 * the paper draws for its kernels (Sec. 3.4, roofline figure), measured
 * rather than taken from a data sheet.  PIC_ERR_ARG for another precision
 * or a NULL output.  Waits. */
pic_status pic_measure_fma_peak(int32_t precision, double* tflops);

/* Message of the calling thread's last failure ("" if none). */
const char* pic_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LIBPIC_PIC_H */
