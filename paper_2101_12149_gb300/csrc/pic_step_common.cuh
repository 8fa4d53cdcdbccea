// Device helpers shared by the forward kernels (pic_kernels.cu) and the
// adjoint kernels (pic_adjoint.cu): kernel arguments, tile-major cell keys,
// gather weights and stencil offsets, the push of one particle, the Esirkepov
// deposit into global memory.  Sharing them makes the adjoint recompute the
// forward step with exactly the forward's arithmetic.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "pic_ctx.h"
#include "pic_device.cuh"

namespace pic {

constexpr int kBlock = 256;

// ---------------------------------------------------------------------------
// cell keys: tile-major, k fastest inside a tile
// ---------------------------------------------------------------------------
__device__ __forceinline__ int key_of(const Geom& g, int i, int j, int k) {
    const int ti = i >> g.lT[0], tj = j >> g.lT[1], tk = k >> g.lT[2];
    const int li = i & (g.T[0] - 1), lj = j & (g.T[1] - 1), lk = k & (g.T[2] - 1);
    const int t = (ti * g.nt[1] + tj) * g.nt[2] + tk;
    const int l = (li << (g.lT[1] + g.lT[2])) | (lj << g.lT[2]) | lk;
    return g.kbase + t * g.cpt + l;
}

__device__ __forceinline__ void tile_origin(const Geom& g, int t, int& oi, int& oj, int& ok) {
    const int tk = t % g.nt[2];
    const int r = t / g.nt[2];
    const int tj = r % g.nt[1];
    const int ti = r / g.nt[1];
    oi = ti << g.lT[0];
    oj = tj << g.lT[1];
    ok = tk << g.lT[2];
}

__device__ __forceinline__ void cell_of(const Geom& g, int key, int& i, int& j, int& k) {
    key -= g.kbase;
    const int lcpt = g.lT[0] + g.lT[1] + g.lT[2];
    const int t = key >> lcpt, l = key & (g.cpt - 1);
    int oi, oj, ok;
    tile_origin(g, t, oi, oj, ok);
    i = oi + (l >> (g.lT[1] + g.lT[2]));
    j = oj + ((l >> g.lT[2]) & (g.T[1] - 1));
    k = ok + (l & (g.T[2] - 1));
}

// Periodic wrap of a position: x >= L -> x - L, x < 0 -> x + L, and a value
// that rounds to L maps to 0.
__device__ __forceinline__ double wrap_pos(double x, double L) {
    if (x >= L) x -= L;
    else if (x < 0.0) x += L;
    if (x >= L) x = 0.0;
    return x;
}

// ---------------------------------------------------------------------------
// kernel arguments
// ---------------------------------------------------------------------------
template <typename R> struct StepArgs {
    Geom g;
    R kq;        // q dt / (2 m)
    R dtc[3];    // dt / d  (FP32-mixed: cell units per unit velocity)
    R jc[3];     // -q / (dt * d_t1 * d_t2): current per unit weight and unit Esirkepov sum
    double dt;
    const R* E[3];
    const R* B[3];
    R* J[3];
    R* pa[7];    // particle arrays (see PartBuf)
    int* key;
    R* old[6];   // split API: old position (3) and displacement (3)
    int* oldkey;
    const int* offsets;
    unsigned* err;
    int* outn;   // outsider count (device)
    int* outl;   // outsider particle indices
    int* cnext;  // when set, count[new key] += 1 for every particle stored (the next sort's histogram)
    const long long* step;
    double drive_amp, drive_k;
    int run;            // tile kernel: particles per lane run (0 = about one cell's worth)
    int pusher;         // 0 Boris, 1 Vay
    int egather;        // 0 momentum-conserving gather, 1 energy-conserving
    float vscale;       // FP32-mixed fixed-point scale of the deposit (largest power of two <= 2^30 / max|coef|)
    float inv_vscale;   // 1 / vscale (a power of two: exact)
    int64_t np;
    const CUtensorMap* tmap;  // batch of boxes: the box's E/B TMA descriptor in global memory, or null
    float g2_fp64;            // FP32-mixed: gamma^2 above which the push's rotation runs in FP64
    // Sorted-order step: the tile kernel reads the particle perm[s] of the
    // source buffer (spa, skey, sid) and writes it to slot s of the current
    // buffer (pa, key, did).  perm == nullptr: in place (the source is the
    // current buffer).
    const int* perm;
    const R* spa[7];
    const int* skey;
    const int* sid;
    int* did;
};

template <typename R> StepArgs<R> make_args(pic_ctx* c) {
    StepArgs<R> a;
    a.g = c->g;
    a.kq = R(c->q * c->dt / (2.0 * c->m));
    for (int d = 0; d < 3; ++d) {
        a.dtc[d] = R(c->dt / c->g.d[d]);
        const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
        a.jc[d] = R(-c->q / (c->dt * c->g.d[t1] * c->g.d[t2]));
        // with the z filter on the particles gather the filtered copy (six
        // arrays of C values in one allocation)
        if (c->filter_passes > 0 && c->Fg) {
            a.E[d] = static_cast<const R*>(c->Fg) + d * c->g.C;
            a.B[d] = static_cast<const R*>(c->Fg) + (3 + d) * c->g.C;
        } else {
            a.E[d] = static_cast<const R*>(c->F[d]);
            a.B[d] = static_cast<const R*>(c->F[3 + d]);
        }
        a.J[d] = static_cast<R*>(c->j_other ? c->Fo[6 + d] : c->F[6 + d]);
    }
    a.dt = c->dt;
    const PartBuf& P = c->P[c->cur];
    for (int i = 0; i < 7; ++i) a.pa[i] = static_cast<R*>(P.a[i]);
    a.key = P.key;
    for (int i = 0; i < 6; ++i) a.old[i] = static_cast<R*>(c->old[i]);
    a.oldkey = c->oldkey;
    a.offsets = c->offsets;
    a.err = c->err;
    a.outn = reinterpret_cast<int*>(c->err + 4);
    a.outl = c->outl;
    a.cnext = c->count_into ? c->count : nullptr;
    a.step = c->d_step;
    a.drive_amp = c->drive_amp;
    a.drive_k = c->drive_k;
    a.pusher = c->pusher;
    a.egather = c->egather;
    // order 1 on the halo-1 layout: runs of two particles over the whole tile
    // (4 % faster than per-warp rows at 2 particles per cell; the shared-memory
    // pipe is not the limit there)
    a.run = c->layout == 2 ? 2 : 0;
    {
        double cmax = 0.0;
        for (int d = 0; d < 3; ++d) {
            const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
            cmax = fmax(cmax, fabs(c->q) * c->w_max / (c->dt * c->g.d[t1] * c->g.d[t2]));
        }
        if (!(cmax > 0.0)) cmax = 1.0;
        int e = 0;
        std::frexp(1073741824.0 / cmax, &e);  // 2^30 / cmax = m 2^e, m in [0.5, 1)
        a.vscale = float(std::ldexp(1.0, e - 1));
        a.inv_vscale = float(std::ldexp(1.0, 1 - e));
    }
    a.np = c->np;
    a.tmap = nullptr;
    a.g2_fp64 = std::isfinite(c->gamma_fp64) ? float(c->gamma_fp64 * c->gamma_fp64) : INFINITY;
    a.perm = nullptr;
    for (int i = 0; i < 7; ++i) a.spa[i] = a.pa[i];
    a.skey = a.key;
    a.sid = P.id;
    a.did = P.id;
    return a;
}

// Arguments of a sorted-order step: the particles come from buffer `src` in
// the order perm gives and go to buffer `dst`.
template <typename R> StepArgs<R> make_args_perm(pic_ctx* c, int src, int dst, const int* perm) {
    StepArgs<R> a = make_args<R>(c);
    const PartBuf& S = c->P[src];
    const PartBuf& D = c->P[dst];
    for (int i = 0; i < 7; ++i) {
        a.spa[i] = static_cast<const R*>(S.a[i]);
        a.pa[i] = static_cast<R*>(D.a[i]);
    }
    a.skey = S.key;
    a.sid = S.id;
    a.key = D.key;
    a.did = D.id;
    a.perm = perm;
    return a;
}

// Arguments of the Yee kernels: E, B, J of one box, its extents, inverse
// cell sizes and the time step h of the update (dt/2 for a B half step).
template <typename R> struct YeeArgs {
    R* E[3];
    R* B[3];
    const R* J[3];
    int n[3];
    R inv[3];
    R h;
    long long* step;  // advanced by one thread when non-null
    int zopen;        // no field beyond the z ends
    int ckc;          // B update with the CKC stencil (cubic cells)
};

// ---------------------------------------------------------------------------
// field sources / current targets: offset tables per axis, plain or wrapped
// ---------------------------------------------------------------------------
template <int P, typename R>
__device__ __forceinline__ R interp(const R* __restrict__ F, const int* ox, const int* oy, const int* oz,
                                    const R* wx, const R* wy, const R* wz) {
    R acc = R(0);
#pragma unroll
    for (int i = 0; i <= P; ++i) {
        R ay = R(0);
#pragma unroll
        for (int j = 0; j <= P; ++j) {
            R az = R(0);
            const R* row = F + ox[i] + oy[j];
#pragma unroll
            for (int k = 0; k <= P; ++k) az += wz[k] * row[oz[k]];
            ay += wy[j] * az;
        }
        acc += wx[i] * ay;
    }
    return acc;
}

// Per-axis gather weights and offsets for node-centred (n) and staggered (s)
// components.  Offsets are element offsets into the source arrays.
template <int P, typename R> struct GatherW {
    R wn[3][P + 1], ws[3][P + 1];
    int on[3][P + 1], os[3][P + 1];
};

// Momentum-conserving gather of E and B (order P along every axis at each
// component's staggered location).
template <int P, typename R>
__device__ __forceinline__ void gather6(const GatherW<P, R>& G, const R* const E[3], const R* const B[3], R EB[6]) {
    EB[0] = interp<P, R>(E[0], G.os[0], G.on[1], G.on[2], G.ws[0], G.wn[1], G.wn[2]);
    EB[1] = interp<P, R>(E[1], G.on[0], G.os[1], G.on[2], G.wn[0], G.ws[1], G.wn[2]);
    EB[2] = interp<P, R>(E[2], G.on[0], G.on[1], G.os[2], G.wn[0], G.wn[1], G.ws[2]);
    EB[3] = interp<P, R>(B[0], G.on[0], G.os[1], G.os[2], G.wn[0], G.ws[1], G.ws[2]);
    EB[4] = interp<P, R>(B[1], G.os[0], G.on[1], G.os[2], G.ws[0], G.wn[1], G.ws[2]);
    EB[5] = interp<P, R>(B[2], G.os[0], G.os[1], G.on[2], G.ws[0], G.ws[1], G.wn[2]);
}

// Weights from the in-cell fractions; offsets either into a staged tile
// (cell at local index l + halo, strides st) or into the global arrays with
// periodic wrap.
// ec: energy-conserving gather (staggered axes at order P - 1).
template <int P, typename R>
__device__ __forceinline__ void gather_weights(const R f[3], GatherW<P, R>& G, int first_n[3], int first_s[3],
                                               bool ec = false) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Shape<P, R>::weights(f[a], first_n[a], G.wn[a]);
        if (ec) staggered_weights_ec<P, R>(f[a], first_s[a], G.ws[a]);
        else staggered_weights<P, R>(f[a], first_s[a], G.ws[a]);
    }
}

template <int P, typename R>
__device__ __forceinline__ void offsets_local(GatherW<P, R>& G, const int base[3], const int st[3],
                                              const int first_n[3], const int first_s[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int r = 0; r <= P; ++r) {
            G.on[a][r] = (base[a] + first_n[a] + r) * st[a];
            G.os[a][r] = (base[a] + first_s[a] + r) * st[a];
        }
}

// With z open, a node beyond the z ends gets weight 0 (and offset 0).
template <int P, typename R>
__device__ __forceinline__ void offsets_global(GatherW<P, R>& G, const Geom& g, const int cell[3],
                                               const int first_n[3], const int first_s[3]) {
    const int st[3] = {g.n[1] * g.n[2], g.n[2], 1};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int r = 0; r <= P; ++r) {
            G.on[a][r] = wrap_once(cell[a] + first_n[a] + r, g.n[a]) * st[a];
            G.os[a][r] = wrap_once(cell[a] + first_s[a] + r, g.n[a]) * st[a];
        }
    if (g.zopen) {
#pragma unroll
        for (int r = 0; r <= P; ++r) {
            if (unsigned(cell[2] + first_n[2] + r) >= unsigned(g.n[2])) G.on[2][r] = 0, G.wn[2][r] = R(0);
            if (unsigned(cell[2] + first_s[2] + r) >= unsigned(g.n[2])) G.os[2][r] = 0, G.ws[2][r] = R(0);
        }
    }
}

// Current target in the global arrays: node (cell + b + slot) per axis,
// wrapped periodically (the "SumBoundary" fold of Sec. 2.4 on one box).
template <int P, typename R> struct JTarget {
    R* J[3];
    int cx, cy, cz;  // first window node per axis (unwrapped)
    int nx, ny, nz;
    int zopen;       // drop current beyond the z ends
    __device__ __forceinline__ void add(int c, int i, int j, int k, R v) const {
        if (zopen && unsigned(cz + k) >= unsigned(nz)) return;
        const int gi = wrap_once(cx + i, nx), gj = wrap_once(cy + j, ny), gk = wrap_once(cz + k, nz);
        atomicAdd(J[c] + ((int64_t)gi * ny + gj) * nz + gk, v);
    }
};

// Esirkepov deposit of one particle: J_c at slot (i,j,k) of the window gets
// coef_c * (sum over the cumulative axis of dS) * Q over the transverse axes,
// Q(a,b) = S0a S0b + dSa S0b/2 + S0a dSb/2 + dSa dSb/3.  The last slot of the
// cumulative sum is zero (sum of dS vanishes) and is not written.
template <int P, typename R>
__device__ __forceinline__ void esirkepov_deposit(const EsirkAxis<P, R>* ax, const R* coef,
                                                  const JTarget<P, R>& t) {
    constexpr int NW = P + 2;
    R A[3][NW], Bq[3][NW];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            A[a][w] = ax[a].S0[w] + R(0.5) * ax[a].dS[w];
            Bq[a][w] = R(0.5) * ax[a].S0[w] + R(1.0 / 3.0) * ax[a].dS[w];
        }
    // J_x: cumulative along x, transverse y, z
    {
        R cum[NW - 1];
        R run = R(0);
#pragma unroll
        for (int w = 0; w < NW - 1; ++w) { run += ax[0].dS[w]; cum[w] = coef[0] * run; }
#pragma unroll
        for (int j = 0; j < NW; ++j)
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const R Q = ax[1].S0[j] * A[2][k] + ax[1].dS[j] * Bq[2][k];
#pragma unroll
                for (int i = 0; i < NW - 1; ++i) t.add(0, i, j, k, cum[i] * Q);
            }
    }
    // J_y: cumulative along y, transverse x, z
    {
        R cum[NW - 1];
        R run = R(0);
#pragma unroll
        for (int w = 0; w < NW - 1; ++w) { run += ax[1].dS[w]; cum[w] = coef[1] * run; }
#pragma unroll
        for (int i = 0; i < NW; ++i)
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const R Q = ax[0].S0[i] * A[2][k] + ax[0].dS[i] * Bq[2][k];
#pragma unroll
                for (int j = 0; j < NW - 1; ++j) t.add(1, i, j, k, cum[j] * Q);
            }
    }
    // J_z: cumulative along z, transverse x, y
    {
        R cum[NW - 1];
        R run = R(0);
#pragma unroll
        for (int w = 0; w < NW - 1; ++w) { run += ax[2].dS[w]; cum[w] = coef[2] * run; }
#pragma unroll
        for (int i = 0; i < NW; ++i)
#pragma unroll
            for (int j = 0; j < NW; ++j) {
                const R Q = ax[0].S0[i] * A[1][j] + ax[0].dS[i] * Bq[1][j];
#pragma unroll
                for (int k = 0; k < NW - 1; ++k) t.add(2, i, j, k, cum[k] * Q);
            }
    }
}

template <int P, typename R>
__device__ __forceinline__ void jtarget_global(JTarget<P, R>& t, const Geom& g, R* const J[3], const int cell[3],
                                               const EsirkAxis<P, R>* ax) {
    for (int c = 0; c < 3; ++c) t.J[c] = J[c];
    t.cx = cell[0] + ax[0].b;
    t.cy = cell[1] + ax[1].b;
    t.cz = cell[2] + ax[2].b;
    t.nx = g.n[0];
    t.ny = g.n[1];
    t.nz = g.n[2];
    t.zopen = g.zopen;
}

// ---------------------------------------------------------------------------
// particle state access (FP64 and FP32-mixed)
// ---------------------------------------------------------------------------
// FP64: positions are global coordinates; cell = floor(x/d), fraction exact.
// x / d, correctly rounded; when d is a normal power of two (unit cells among
// them) by the exact reciprocal, which avoids the FP64 division.
__device__ __forceinline__ double div_by_cell(double x, double d) {
    const long long b = __double_as_longlong(d);
    if ((b & 0x000FFFFFFFFFFFFFll) == 0 && b > 0x0010000000000000ll && b < 0x7FE0000000000000ll)
        return x * __longlong_as_double(0x7FE0000000000000ll - b);
    return x / d;
}

__device__ __forceinline__ void split_pos(double x, double d, int n, int& cell, double& f) {
    const double p = div_by_cell(x, d);
    double fl = floor(p);
    int c = int(fl);
    if (c >= n) c = n - 1, fl = double(n - 1);
    if (c < 0) c = 0, fl = 0.0;
    cell = c;
    f = p - fl;
}

// One particle through gather, push and advance.  `f0` is the fraction
// inside the old cell, `f1` the new position relative to the old cell (cell
// units).  For FP64 the advance is done in global coordinates with the same
// operation order as the definition (x += (dt u) / gamma), then f1 follows
// exactly from the new global position.
template <typename R> struct Moved {
    R u[3];
    R f0[3], f1[3];
    double xg1[3];  // FP64: unwrapped new global position
    bool ok;
};

template <int P, typename R>
__device__ __forceinline__ void push_particle(const StepArgs<R>& A, R EB[6], const int cell[3], const R f0[3],
                                              const double xg0[3], R u[3], Moved<R>& mv) {
    if (A.drive_amp != 0.0) {
        const double t = double(*A.step) * A.dt;
        const double xp = sizeof(R) == 8 ? xg0[0] : (double(cell[0]) + double(f0[0])) * A.g.d[0];
        EB[1] += R(A.drive_amp * cos(A.drive_k * xp - A.drive_k * t));
    }
    if (A.pusher) vay<R>(A.kq, EB, EB + 3, u, A.g2_fp64);
    else boris<R>(A.kq, EB, EB + 3, u, A.g2_fp64);
    mv.ok = true;
    if (sizeof(R) == 8) {
        const double gi = 1.0 / sqrt(1.0 + double(u[0]) * double(u[0]) + double(u[1]) * double(u[1]) +
                                     double(u[2]) * double(u[2]));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double dx = __dmul_rn(__dmul_rn(A.dt, double(u[a])), gi);
            mv.xg1[a] = __dadd_rn(xg0[a], dx);
            const double p1 = div_by_cell(mv.xg1[a], A.g.d[a]);
            mv.f1[a] = R(p1 - double(cell[a]));
            mv.f0[a] = f0[a];
            if (!(fabs(double(mv.f1[a] - f0[a])) < 1.0)) mv.ok = false;
        }
    } else {
        const R gi = R(1) / sqrt_<R>(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mv.f0[a] = f0[a];
            mv.f1[a] = f0[a] + A.dtc[a] * u[a] * gi;
            mv.xg1[a] = 0.0;
            if (!(fabsf(float(mv.f1[a] - f0[a])) < 1.0f)) mv.ok = false;
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) mv.u[a] = u[a];
}

// New cell and fraction of a move, FP32-mixed: cell += floor(f1), f -= floor(f1),
// cell wrapped periodically.
__device__ __forceinline__ void renormalise(float f1, int cell, int n, int& ncell, float& nf) {
    const float fl = floorf(f1);
    float f = f1 - fl;
    int c = cell + int(fl);
    if (f >= 1.0f) { f -= 1.0f; c += 1; }
    ncell = wrap_once(c, n);
    nf = f;
}

// Load a particle's cell, in-cell fraction, momentum and weight.
template <typename R>
__device__ __forceinline__ void load_particle(const StepArgs<R>& A, int p, int cell[3], R f0[3], double xg0[3],
                                              R u[3], R& wq) {
    const Geom& g = A.g;
    if (sizeof(R) == 8) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xg0[a] = double(A.pa[a][p]);
            double f;
            split_pos(xg0[a], g.d[a], g.n[a], cell[a], f);
            f0[a] = R(f);
        }
    } else {
        cell_of(g, A.key[p], cell[0], cell[1], cell[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            f0[a] = A.pa[a][p];
            xg0[a] = 0.0;
        }
    }
    u[0] = A.pa[3][p];
    u[1] = A.pa[4][p];
    u[2] = A.pa[5][p];
    wq = A.pa[6][p];
}

// A particle's stored data as loaded (key and the 7 reals), so that the tile
// kernel can issue the next particle's loads before it works on the current one.
template <typename R> struct RawParticle {
    int key;
    int id;  // sorted-order step only
    R a[7];
};

// Particle in slot s of the step's order: slot s of the current buffer, or
// particle perm[s] of the source buffer in a sorted-order step.
template <typename R> __device__ __forceinline__ void load_raw(const StepArgs<R>& A, int s, RawParticle<R>& r) {
    const int p = A.perm ? A.perm[s] : s;
    r.key = (sizeof(R) == 4 || A.perm) ? A.skey[p] : 0;
    r.id = A.perm ? A.sid[p] : 0;
#pragma unroll
    for (int i = 0; i < 7; ++i) r.a[i] = A.spa[i][p];
}

// A particle written back unchanged (a rejected move) into slot s: only a
// sorted-order step has to copy it, in place it is already there.
template <typename R> __device__ __forceinline__ void keep_particle(const StepArgs<R>& A, int s, const RawParticle<R>& r) {
    if (A.cnext) atomicAdd(A.cnext + (A.perm ? r.key : A.key[s]), 1);
    if (!A.perm) return;
#pragma unroll
    for (int i = 0; i < 7; ++i) A.pa[i][s] = r.a[i];
    A.key[s] = r.key;
    A.did[s] = r.id;
}

// load_particle on data already loaded.
template <typename R>
__device__ __forceinline__ void decode_particle(const StepArgs<R>& A, const RawParticle<R>& r, int cell[3], R f0[3],
                                                double xg0[3], R u[3], R& wq) {
    const Geom& g = A.g;
    if (sizeof(R) == 8) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xg0[a] = double(r.a[a]);
            double f;
            split_pos(xg0[a], g.d[a], g.n[a], cell[a], f);
            f0[a] = R(f);
        }
    } else {
        cell_of(g, r.key, cell[0], cell[1], cell[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            f0[a] = r.a[a];
            xg0[a] = 0.0;
        }
    }
    u[0] = r.a[3];
    u[1] = r.a[4];
    u[2] = r.a[5];
    wq = r.a[6];
}

// Store the moved particle in place: momentum, wrapped position, new cell key.
// With z open, a particle whose new z is outside [0, Lz) gets the removed key.
template <typename R>
__device__ __forceinline__ void store_particle(const StepArgs<R>& A, int p, const int cell[3], const Moved<R>& mv) {
    const Geom& g = A.g;
#pragma unroll
    for (int a = 0; a < 3; ++a) A.pa[3 + a][p] = mv.u[a];
    int nc[3];
    bool gone = false;
    if (sizeof(R) == 8) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double xw = mv.xg1[a];
            if (a == 2 && g.zopen) gone = !(xw >= 0.0 && xw < g.L[2]);
            else xw = wrap_pos(xw, g.L[a]);
            A.pa[a][p] = R(xw);
            double f;
            split_pos(xw, g.d[a], g.n[a], nc[a], f);
        }
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float nf;
            if (a == 2 && g.zopen) {
                const float fl = floorf(float(mv.f1[2]));
                nf = float(mv.f1[2]) - fl;
                int cz = cell[2] + int(fl);
                if (nf >= 1.0f) nf -= 1.0f, cz += 1;
                gone = unsigned(cz) >= unsigned(g.n[2]);
                nc[2] = gone ? 0 : cz;
            } else {
                renormalise(float(mv.f1[a]), cell[a], g.n[a], nc[a], nf);
            }
            A.pa[a][p] = R(nf);
        }
    }
    const int nkey = gone ? dead_key(g) : key_of(g, nc[0], nc[1], nc[2]);
    A.key[p] = nkey;
    if (A.cnext) atomicAdd(A.cnext + nkey, 1);
}

// Gather + push + advance + Esirkepov for one tile of cells per CTA.
// Particles whose cell is not in the tile (possible only between sorts) are
// appended to the outsider list and left for k_outsiders.
}  // namespace pic
