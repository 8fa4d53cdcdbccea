// Particle and field kernels of libpic (sm_103a).
//
//  k_tile_step      fused gather + Boris + advance + Esirkepov for one tile
//                   of cells per CTA: E/B of the tile and its halo staged in
//                   shared memory, J accumulated in shared memory, one
//                   vectorised atomic flush per tile (Sec. 3.1 fuses gather
//                   and push; Sec. 3.4 discusses shared-memory buffers).
//  k_gather_push    one particle per thread, fields read from global memory.
//  k_deposit        one particle per thread, Esirkepov with global atomics
//                   (the paper's GPU deposit, Sec. 3.4.1).
//  k_yee_b/k_yee_e  Yee FDTD half-step of B / full step of E (Sec. 2.4).
//  conversions, particle load/store, diagnostics.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <type_traits>

#include "pic_ctx.h"
#include "pic_device.cuh"
#include "pic_step_common.cuh"

namespace pic {

// ---------------------------------------------------------------------------
// fused tile kernel
// ---------------------------------------------------------------------------
// Shared-memory boxes of one tile, sized for the largest tile of the layout
// (MX x MY x MZ cells); smaller tiles use the low corner, so every stride is a
// compile-time constant and each shared access is base + immediate.
//   E/B box: cells [-2, T+2) per axis, z rows of pitch EP
//   J box:   x, y [-2, T+3), z [-4, T+4), z rows of pitch JP (z padded so the
//            flush moves aligned float4s)
// Two layouts.  4 x 4 x 32 when nz is a multiple of 32: the lanes of a warp
// take 32 consecutive cells in tile order (one z-row, or the end of one and
// the start of the next), and with row and plane pitches that are multiples
// of 32 words the bank of every access is its z index, so gathers and
// deposits hit 32 distinct banks whatever the per-lane staggering offsets.
// Otherwise up to 8 x 8 x 8 cells.
template <int MX, int MY, int MZ, int EP, int JP> struct Layout {
    static constexpr int EX = MX + 4, EY = MY + 4, EZ = MZ + 4;
    static constexpr int eY = EP, eX = EY * EP, eVol = EX * EY * EP;
    static constexpr int JX = MX + 5, JY = MY + 5, JZ = MZ + 8;
    static constexpr int jY = JP, jX = JY * JP, jVol = JX * JY * JP;
    static_assert(EP >= EZ && JP >= JZ && JP % 4 == 0, "row pitches");
    // FP64: J box of doubles (3 components); FP32-mixed: J box of fixed-point
    // (lo, hi) int32 pairs (3 components x 2 arrays)
    template <typename R> static constexpr size_t smem_bytes() {
        return sizeof(R) == 8 ? 8 * (6 * size_t(eVol) + 3 * size_t(jVol)) : 4 * (6 * size_t(eVol) + 6 * size_t(jVol));
    }
};
// FP64 keeps compact pitches: the bank-conflict-free ones would not fit its
// shared memory, and the FP64 path is bound by FP64 arithmetic.
template <typename R>
using LayoutRow = std::conditional_t<sizeof(R) == 4, Layout<4, 4, 32, 64, 64>, Layout<4, 4, 32, 36, 40>>;
using LayoutCube = Layout<8, 8, 8, 12, 20>;

// Gather of one component from the staged box: `base` points at the first
// stencil node.
template <int P, typename R, class LY>
__device__ __forceinline__ R interp_smem(const R* __restrict__ base, const R* wx, const R* wy, const R* wz) {
    R acc = R(0);
#pragma unroll
    for (int i = 0; i <= P; ++i) {
        R ay = R(0);
#pragma unroll
        for (int j = 0; j <= P; ++j) {
            R az = R(0);
#pragma unroll
            for (int k = 0; k <= P; ++k) az += wz[k] * base[i * LY::eX + j * LY::eY + k];
            ay += wy[j] * az;
        }
        acc += wx[i] * ay;
    }
    return acc;
}

// Esirkepov deposit of one particle into the staged J box; `base` is the
// element offset of window slot (0,0,0).  Same arithmetic as
// esirkepov_deposit (the global-memory form).
template <int P, typename R, class LY, int NC = P + 1, int NT = P + 2>
__device__ __forceinline__ void esirkepov_smem(R* __restrict__ J0, R* __restrict__ J1, R* __restrict__ J2, int base,
                                               const EsirkAxis<P, R> ax[3], const R coef[3]) {
    R* jx = J0 + base;
    R* jy = J1 + base;
    R* jz = J2 + base;
    {
        R cum[NC];
        R run = R(0);
#pragma unroll
        for (int w = 0; w < NC; ++w) { run += ax[0].dS[w]; cum[w] = coef[0] * run; }
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int k = 0; k < NT; ++k) {
                const R Az = ax[2].S0[k] + R(0.5) * ax[2].dS[k];
                const R Bz = R(0.5) * ax[2].S0[k] + R(1.0 / 3.0) * ax[2].dS[k];
                const R Q = ax[1].S0[j] * Az + ax[1].dS[j] * Bz;
#pragma unroll
                for (int i = 0; i < NC; ++i) atomicAdd(jx + i * LY::jX + j * LY::jY + k, cum[i] * Q);
            }
    }
    {
        R cum[NC];
        R run = R(0);
#pragma unroll
        for (int w = 0; w < NC; ++w) { run += ax[1].dS[w]; cum[w] = coef[1] * run; }
#pragma unroll
        for (int i = 0; i < NT; ++i)
#pragma unroll
            for (int k = 0; k < NT; ++k) {
                const R Az = ax[2].S0[k] + R(0.5) * ax[2].dS[k];
                const R Bz = R(0.5) * ax[2].S0[k] + R(1.0 / 3.0) * ax[2].dS[k];
                const R Q = ax[0].S0[i] * Az + ax[0].dS[i] * Bz;
#pragma unroll
                for (int j = 0; j < NC; ++j) atomicAdd(jy + i * LY::jX + j * LY::jY + k, cum[j] * Q);
            }
    }
    {
        R cum[NC];
        R run = R(0);
#pragma unroll
        for (int w = 0; w < NC; ++w) { run += ax[2].dS[w]; cum[w] = coef[2] * run; }
#pragma unroll
        for (int i = 0; i < NT; ++i)
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const R Ay = ax[1].S0[j] + R(0.5) * ax[1].dS[j];
                const R By = R(0.5) * ax[1].S0[j] + R(1.0 / 3.0) * ax[1].dS[j];
                const R Q = ax[0].S0[i] * Ay + ax[0].dS[i] * By;
#pragma unroll
                for (int k = 0; k < NC; ++k) atomicAdd(jz + i * LY::jX + j * LY::jY + k, cum[k] * Q);
            }
    }
}

// FP32-mixed deposit into the staged J box in exact fixed point.
//
// Every Esirkepov contribution obeys |v| <= |coef|: the cumulative sum of dS
// is a difference of two cumulative shape distributions, bounded by the move
// (< 1 cell), and Q <= 1.  With vscale = 2^30 / max|coef|, x = rn(v vscale)
// fits in 31 bits; it is split as x = hi 2^15 + lo (hi = x rounded to a
// multiple of 2^15, |lo| <= 2^14) and the halves go to two int32 arrays by
// native shared-memory integer reductions.  Integer sums are exact and
// independent of order; with at most 65535 particles per tile neither sum
// can overflow (65535 * 2^15 < 2^31).  The flush rebuilds hi 2^15 + lo.
__device__ __forceinline__ void red_fixed(int* lo, int* hi, float v, float vscale) {
    const int x = __float2int_rn(v * vscale);
    const int h = (x + (1 << 14)) >> 15;
    const int l = x - (h << 15);
    atomicAdd(lo, l);
    atomicAdd(hi, h);
}

template <int P, class LY, int NC = P + 1, int NT = P + 2>
__device__ __forceinline__ void esirkepov_smem_fixed(int* __restrict__ sJ, int base, const EsirkAxis<P, float> ax[3],
                                                     const float coef[3], float vscale) {
    int* jx = sJ + base;                  // lo of J_x; hi at + jVol
    int* jy = sJ + 2 * LY::jVol + base;   // lo of J_y
    int* jz = sJ + 4 * LY::jVol + base;   // lo of J_z
    constexpr int H = LY::jVol;
    {
        float cum[NC];
        float run = 0.f;
#pragma unroll
        for (int w = 0; w < NC; ++w) { run += ax[0].dS[w]; cum[w] = coef[0] * run; }
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int kk = 0; kk < NT; ++kk) {
                const float Az = ax[2].S0[kk] + 0.5f * ax[2].dS[kk];
                const float Bz = 0.5f * ax[2].S0[kk] + (1.0f / 3.0f) * ax[2].dS[kk];
                const float Q = ax[1].S0[j] * Az + ax[1].dS[j] * Bz;
#pragma unroll
                for (int i = 0; i < NC; ++i) {
                    const int o = i * LY::jX + j * LY::jY + kk;
                    red_fixed(jx + o, jx + H + o, cum[i] * Q, vscale);
                }
            }
    }
    {
        float cum[NC];
        float run = 0.f;
#pragma unroll
        for (int w = 0; w < NC; ++w) { run += ax[1].dS[w]; cum[w] = coef[1] * run; }
#pragma unroll
        for (int i = 0; i < NT; ++i)
#pragma unroll
            for (int kk = 0; kk < NT; ++kk) {
                const float Az = ax[2].S0[kk] + 0.5f * ax[2].dS[kk];
                const float Bz = 0.5f * ax[2].S0[kk] + (1.0f / 3.0f) * ax[2].dS[kk];
                const float Q = ax[0].S0[i] * Az + ax[0].dS[i] * Bz;
#pragma unroll
                for (int j = 0; j < NC; ++j) {
                    const int o = i * LY::jX + j * LY::jY + kk;
                    red_fixed(jy + o, jy + H + o, cum[j] * Q, vscale);
                }
            }
    }
    {
        float cum[NC];
        float run = 0.f;
#pragma unroll
        for (int w = 0; w < NC; ++w) { run += ax[2].dS[w]; cum[w] = coef[2] * run; }
#pragma unroll
        for (int i = 0; i < NT; ++i)
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const float Ay = ax[1].S0[j] + 0.5f * ax[1].dS[j];
                const float By = 0.5f * ax[1].S0[j] + (1.0f / 3.0f) * ax[1].dS[j];
                const float Q = ax[0].S0[i] * Ay + ax[0].dS[i] * By;
#pragma unroll
                for (int kk = 0; kk < NC; ++kk) {
                    const int o = i * LY::jX + j * LY::jY + kk;
                    red_fixed(jz + o, jz + H + o, cum[kk] * Q, vscale);
                }
            }
    }
}

// Deposit of one particle into the staged J box: the window's first node is
// (li + 2 + b_x, lj + 2 + b_y, lk + 4 + b_z) in box coordinates.  NARROW: all
// three axes have both shapes starting at node b, so the stencil is P cumulative
// slots by (P + 1)^2 transverse nodes (the skipped slots hold exact zeros and,
// on the cumulative axis, the rounding residue of sum dS = 0).
template <int P, typename R, class LY, bool NARROW>
__device__ __forceinline__ void tile_deposit(const StepArgs<R>& A, R* sJ, int li, int lj, int lk,
                                             const EsirkAxis<P, R> ax[3], R wq) {
    constexpr int NC = NARROW ? P : P + 1;
    constexpr int NT = NARROW ? P + 1 : P + 2;
    const R coef[3] = {A.jc[0] * wq, A.jc[1] * wq, A.jc[2] * wq};
    const int bx = li + 2 + ax[0].b, by = lj + 2 + ax[1].b, bz = lk + 4 + ax[2].b;
    PIC_CHECK_OR(bx >= 0 && bx + P + 1 < LY::JX && by >= 0 && by + P + 1 < LY::JY && bz >= 0 && bz + P + 1 < LY::JZ,
                 A.err, 4, ((long long)(ax[0].b + 8) << 16) | ((ax[1].b + 8) << 8) | (ax[2].b + 8), return);
    const int base = bx * LY::jX + by * LY::jY + bz;
    if constexpr (sizeof(R) == 4)
        esirkepov_smem_fixed<P, LY, NC, NT>(reinterpret_cast<int*>(sJ), base,
                                            reinterpret_cast<const EsirkAxis<P, float>*>(ax),
                                            reinterpret_cast<const float*>(coef), A.vscale);
    else
        esirkepov_smem<P, R, LY, NC, NT>(sJ, sJ + LY::jVol, sJ + 2 * LY::jVol, base, ax, coef);
}

// Position of the n-th set bit (n counted from 0) of m; n < popcount(m).
__device__ __forceinline__ int nth_set_bit(unsigned m, int n) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const unsigned low = (1u << w) - 1u;
        const int c = __popc(m & low);
        if (n >= c) {
            n -= c;
            m >>= w;
            pos += w;
        } else {
            m &= low;
        }
    }
    return pos;
}

// A move waiting for the full-window deposit: local cell, the in-cell
// fractions before and after (relative to the old cell) and the weight.
template <typename R> struct TileMove {
    R f0[3], f1[3], wq;
    int cell;  // li | lj << 8 | lk << 16
    __device__ __forceinline__ static TileMove zero() {
        TileMove t;
#pragma unroll
        for (int a = 0; a < 3; ++a) t.f0[a] = t.f1[a] = R(0);
        t.wq = R(0);
        t.cell = 0;
        return t;
    }
    __device__ __forceinline__ void set(int li, int lj, int lk, const R* a0, const R* a1, R w) {
#pragma unroll
        for (int a = 0; a < 3; ++a) f0[a] = a0[a], f1[a] = a1[a];
        wq = w;
        cell = li | (lj << 8) | (lk << 16);
    }
    __device__ __forceinline__ TileMove shfl(int src) const {
        TileMove t;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            t.f0[a] = __shfl_sync(0xffffffffu, f0[a], src);
            t.f1[a] = __shfl_sync(0xffffffffu, f1[a], src);
        }
        t.wq = __shfl_sync(0xffffffffu, wq, src);
        t.cell = __shfl_sync(0xffffffffu, cell, src);
        return t;
    }
    template <int P, class LY> __device__ __forceinline__ void deposit(const StepArgs<R>& A, R* sJ) const {
        EsirkAxis<P, R> ax[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) ax[a].init(f0[a], f1[a]);
        tile_deposit<P, R, LY, false>(A, sJ, cell & 0xff, (cell >> 8) & 0xff, cell >> 16, ax, wq);
    }
};

// Block size of the tile kernel: FP32-mixed 512 threads (one CTA per SM, its
// shared memory holding the fixed-point J box), FP64 256.
template <typename R> constexpr int tile_block() { return sizeof(R) == 4 ? 512 : 256; }

// One tile t of the box described by A, by the whole CTA; `smem_raw` is the
// CTA's dynamic shared memory.  Returns with the block converged.
template <int P, typename R, class LY>
__device__ __forceinline__ void tile_body(const StepArgs<R>& A, const int t, unsigned char* smem_raw) {
    R* sm = reinterpret_cast<R*>(smem_raw);
    const Geom& g = A.g;
    constexpr bool kFixed = sizeof(R) == 4;
    R* sEB = sm;                  // 6 * eVol
    R* sJ = sm + 6 * LY::eVol;    // FP64: 3 * jVol doubles; FP32-mixed: 6 * jVol int32 (lo, hi per component)
    int* sJi = reinterpret_cast<int*>(sJ);

    const int beg = A.offsets[(int64_t)t * g.cpt];
    const int end = A.offsets[(int64_t)(t + 1) * g.cpt];
    if (end <= beg) return;
    PIC_CHECK_OR(beg >= 0 && end <= A.np, A.err, 1, ((long long)beg << 32) | unsigned(end), return);
    int oi, oj, ok;
    tile_origin(g, t, oi, oj, ok);

    // stage E, B of the tile and a halo of 2 (wrapped)
    {
        const int ex = g.T[0] + 4, ey = g.T[1] + 4, ez = g.T[2] + 4;
        const int vol = ex * ey * ez;
        for (int e = threadIdx.x; e < 6 * vol; e += blockDim.x) {
            const int c = e / vol;
            int r = e - c * vol;
            const int a = r / (ey * ez);
            r -= a * ey * ez;
            const int b = r / ez;
            const int kk = r - b * ez;
            const int gi = wrap_any(oi - 2 + a, g.n[0]);
            const int gj = wrap_any(oj - 2 + b, g.n[1]);
            const int kz = ok - 2 + kk;
            R v = R(0);
            if (!g.zopen || unsigned(kz) < unsigned(g.n[2])) {  // z open: nothing beyond the ends
                const int gk = wrap_any(kz, g.n[2]);
                const int64_t gidx = ((int64_t)gi * g.n[1] + gj) * g.n[2] + gk;
                PIC_CHECK_OR(gidx >= 0 && gidx < g.C && a < LY::EX && b < LY::EY && kk < LY::EZ, A.err, 2, gidx,
                             continue);
                v = c < 3 ? A.E[c][gidx] : A.B[c - 3][gidx];
            }
            sEB[c * LY::eVol + a * LY::eX + b * LY::eY + kk] = v;
        }
        if (kFixed)
            for (int e = threadIdx.x; e < 6 * LY::jVol; e += blockDim.x) sJi[e] = 0;
        else
            for (int e = threadIdx.x; e < 3 * LY::jVol; e += blockDim.x) sJ[e] = R(0);
    }
    __syncthreads();

    // The tile's particles are cell-sorted; consecutive lanes take consecutive
    // runs of about one cell's worth of particles, so the lanes of a warp work
    // in neighbouring cells (distinct shared-memory banks).
    const int cnt = end - beg;
    const int run = A.run > 0 ? A.run : max(1, (cnt + (g.cpt >> 1)) / g.cpt);
    const int nrun = (cnt + run - 1) / run;
    // Warps step their lanes' runs in lockstep.  A move whose old and new
    // shapes start on the same node along every axis (most moves: crossing a
    // cell face is rare) deposits the narrow stencil at once; the others go to
    // a per-warp queue held one slot per lane in registers and are deposited
    // 32 at a time with the full window, so neither kind runs with idle lanes.
    const int lane = threadIdx.x & 31;
    TileMove<R> qs = TileMove<R>::zero();  // this lane's queue slot
    int qn = 0;                            // queued moves (warp-uniform)
    for (int rbase = threadIdx.x - lane; rbase < nrun; rbase += blockDim.x) {
        const int rr = rbase + lane;
        const int p0 = beg + rr * run;
        const int len = rr < nrun ? min(run, end - p0) : 0;
        const int maxlen = __reduce_max_sync(0xffffffffu, len);
        for (int it = 0; it < maxlen; ++it) {
            const int p = p0 + it;
            bool wide = false;
            TileMove<R> mine = TileMove<R>::zero();
            if (it < len) {
                int cell[3];
                R f0[3], u[3], wq;
                double xg0[3];
                load_particle<R>(A, p, cell, f0, xg0, u, wq);
                const int li = cell[0] - oi, lj = cell[1] - oj, lk = cell[2] - ok;
                // the fixed-point sums are exact for up to 65535 particles per tile
                const bool inside = unsigned(li) < unsigned(g.T[0]) && unsigned(lj) < unsigned(g.T[1]) &&
                                    unsigned(lk) < unsigned(g.T[2]) && (!kFixed || p - beg < 65535);
                if (!inside) {
                    const int slot = atomicAdd(A.outn, 1);
                    A.outl[slot] = p;
                } else {
                    R EB[6];
                    {
                        GatherW<P, R> G;
                        int fn[3], fs[3];
                        gather_weights<P, R>(f0, G, fn, fs);
                        const int bnx = (li + 2 + fn[0]) * LY::eX, bsx = (li + 2 + fs[0]) * LY::eX;
                        const int bny = (lj + 2 + fn[1]) * LY::eY, bsy = (lj + 2 + fs[1]) * LY::eY;
                        const int bnz = lk + 2 + fn[2], bsz = lk + 2 + fs[2];
                        EB[0] = interp_smem<P, R, LY>(sEB + 0 * LY::eVol + bsx + bny + bnz, G.ws[0], G.wn[1], G.wn[2]);
                        EB[1] = interp_smem<P, R, LY>(sEB + 1 * LY::eVol + bnx + bsy + bnz, G.wn[0], G.ws[1], G.wn[2]);
                        EB[2] = interp_smem<P, R, LY>(sEB + 2 * LY::eVol + bnx + bny + bsz, G.wn[0], G.wn[1], G.ws[2]);
                        EB[3] = interp_smem<P, R, LY>(sEB + 3 * LY::eVol + bnx + bsy + bsz, G.wn[0], G.ws[1], G.ws[2]);
                        EB[4] = interp_smem<P, R, LY>(sEB + 4 * LY::eVol + bsx + bny + bsz, G.ws[0], G.wn[1], G.ws[2]);
                        EB[5] = interp_smem<P, R, LY>(sEB + 5 * LY::eVol + bsx + bsy + bnz, G.ws[0], G.ws[1], G.wn[2]);
                    }
                    Moved<R> mv;
                    push_particle<P, R>(A, EB, cell, f0, xg0, u, mv);
                    if (!mv.ok) {
                        raise_error(A.err, ERRBIT_PARTICLE);
                    } else {
                        store_particle<R>(A, p, cell, mv);
                        EsirkAxis<P, R> ax[3];
#pragma unroll
                        for (int a = 0; a < 3; ++a) ax[a].init(mv.f0[a], mv.f1[a]);
                        if (ax[0].narrow && ax[1].narrow && ax[2].narrow) {
                            tile_deposit<P, R, LY, true>(A, sJ, li, lj, lk, ax, wq);
                        } else {
                            wide = true;
                            mine.set(li, lj, lk, mv.f0, mv.f1, wq);
                        }
                    }
                }
            }
            const unsigned wm = __ballot_sync(0xffffffffu, wide);
            if (wm == 0u) continue;
            // queue the full-window moves: slots qn, qn+1, ... pull from the k-th wide lane
            const int nw = __popc(wm);
            const int take = min(nw, 32 - qn);
            {
                const int r = lane - qn;
                const bool recv = r >= 0 && r < take;
                const TileMove<R> got = mine.shfl(recv ? nth_set_bit(wm, r) : lane);
                if (recv) qs = got;
            }
            qn += take;
            if (qn == 32) {
                qs.template deposit<P, LY>(A, sJ);
                qn = nw - take;
                if (qn > 0) {
                    const bool recv = lane < qn;
                    const TileMove<R> got = mine.shfl(recv ? nth_set_bit(wm, take + lane) : lane);
                    if (recv) qs = got;
                }
            }
        }
    }
    if (lane < qn) qs.template deposit<P, LY>(A, sJ);
    __syncthreads();

    // flush the tile's current into the global arrays (periodic fold)
    const int jx = g.T[0] + 5, jy = g.T[1] + 5, jz = g.T[2] + 8;
    if (kFixed && (g.T[2] % 4) == 0 && (g.n[2] % 4) == 0) {
        const int q4 = jz / 4;
        const int rows = jx * jy;
        for (int e = threadIdx.x; e < 3 * rows * q4; e += blockDim.x) {
            const int c = e / (rows * q4);
            int r = e - c * rows * q4;
            const int row = r / q4;
            const int q = r - row * q4;
            const int a = row / jy;
            const int b = row - a * jy;
            const int o = 2 * c * LY::jVol + a * LY::jX + b * LY::jY + 4 * q;
            const int4 lo = *reinterpret_cast<const int4*>(sJi + o);
            const int4 hi = *reinterpret_cast<const int4*>(sJi + o + LY::jVol);
            if ((lo.x | lo.y | lo.z | lo.w | hi.x | hi.y | hi.z | hi.w) == 0) continue;
            const float4 v = make_float4(float(double((long long)hi.x * 32768 + lo.x) * A.inv_vscale),
                                         float(double((long long)hi.y * 32768 + lo.y) * A.inv_vscale),
                                         float(double((long long)hi.z * 32768 + lo.z) * A.inv_vscale),
                                         float(double((long long)hi.w * 32768 + lo.w) * A.inv_vscale));
            const int gi = wrap_any(oi - 2 + a, g.n[0]);
            const int gj = wrap_any(oj - 2 + b, g.n[1]);
            // a group of 4 starts at a multiple of 4 and nz % 4 == 0: it is all inside or all beyond the z ends
            if (g.zopen && unsigned(ok - 4 + 4 * q) >= unsigned(g.n[2])) continue;
            const int gk = wrap_any(ok - 4 + 4 * q, g.n[2]);
            PIC_CHECK_OR(gk + 3 < g.n[2] && ((gk & 3) == 0), A.err, 6, gk, continue);
            float* dst = reinterpret_cast<float*>(A.J[c]) + ((int64_t)gi * g.n[1] + gj) * g.n[2] + gk;
            atomicAdd(reinterpret_cast<float4*>(dst), v);
        }
    } else {
        const int vol = jx * jy * jz;
        for (int e = threadIdx.x; e < 3 * vol; e += blockDim.x) {
            const int c = e / vol;
            int r = e - c * vol;
            const int a = r / (jy * jz);
            r -= a * jy * jz;
            const int b = r / jz;
            const int kk = r - b * jz;
            const int o = a * LY::jX + b * LY::jY + kk;
            R v;
            if (kFixed)
                v = R(double((long long)sJi[2 * c * LY::jVol + LY::jVol + o] * 32768 + sJi[2 * c * LY::jVol + o]) *
                      A.inv_vscale);
            else
                v = sJ[c * LY::jVol + o];
            if (v == R(0)) continue;
            if (g.zopen && unsigned(ok - 4 + kk) >= unsigned(g.n[2])) continue;
            const int gi = wrap_any(oi - 2 + a, g.n[0]);
            const int gj = wrap_any(oj - 2 + b, g.n[1]);
            const int gk = wrap_any(ok - 4 + kk, g.n[2]);
            atomicAdd(A.J[c] + ((int64_t)gi * g.n[1] + gj) * g.n[2] + gk, v);
        }
    }
}

template <int P, typename R, class LY>
__global__ void __launch_bounds__(tile_block<R>(), 1) k_tile_step(StepArgs<R> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_body<P, R, LY>(A, int(blockIdx.x), smem_raw);
}

// Batch of boxes: a persistent grid pulls (box, tile) items from a queue
// counter (zeroed before the launch); each item's box arguments are copied
// into shared memory first.  Items are ordered heaviest first.
template <int P, typename R, class LY>
__global__ void __launch_bounds__(tile_block<R>(), 1)
    k_tile_step_batch(const StepArgs<R>* __restrict__ boxes, const int2* __restrict__ items, int nitems, int* queue) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) StepArgs<R> sA;
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int2 bt = items[it];
        {
            const int* src = reinterpret_cast<const int*>(boxes + bt.x);
            int* dst = reinterpret_cast<int*>(&sA);
            for (int w = threadIdx.x; w < int(sizeof(StepArgs<R>) / 4); w += blockDim.x) dst[w] = src[w];
        }
        __syncthreads();
        tile_body<P, R, LY>(sA, bt.y, smem_raw);
        __syncthreads();
    }
}

// One particle the tile kernel listed as outside its tile: gather from global
// memory, push, deposit with global atomics (the same arithmetic).
template <int P, typename R>
__device__ __forceinline__ void outsider_body(const StepArgs<R>& A, const int p) {
    int cell[3];
    R f0[3], u[3], wq;
    double xg0[3];
    load_particle<R>(A, p, cell, f0, xg0, u, wq);
    R EB[6];
    {
        GatherW<P, R> G;
        int fn[3], fs[3];
        gather_weights<P, R>(f0, G, fn, fs);
        offsets_global<P, R>(G, A.g, cell, fn, fs);
        gather6<P, R>(G, A.E, A.B, EB);
    }
    Moved<R> mv;
    push_particle<P, R>(A, EB, cell, f0, xg0, u, mv);
    if (!mv.ok) {
        raise_error(A.err, ERRBIT_PARTICLE);
        return;
    }
    EsirkAxis<P, R> ax[3];
    for (int a = 0; a < 3; ++a) ax[a].init(mv.f0[a], mv.f1[a]);
    const R coef[3] = {A.jc[0] * wq, A.jc[1] * wq, A.jc[2] * wq};
    JTarget<P, R> jt;
    jtarget_global<P, R>(jt, A.g, A.J, cell, ax);
    esirkepov_deposit<P, R>(ax, coef, jt);
    store_particle<R>(A, p, cell, mv);
}

template <int P, typename R>
__global__ void __launch_bounds__(kBlock) k_outsiders(StepArgs<R> A) {
    const int n = *A.outn;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        outsider_body<P, R>(A, A.outl[i]);
}

// Batch: the box of an outsider is found from the boxes' first particle
// indices (pbase, nboxes + 1 entries, ascending).
template <int P, typename R>
__global__ void __launch_bounds__(kBlock)
    k_outsiders_batch(const StepArgs<R>* __restrict__ boxes, const int64_t* __restrict__ pbase, int nboxes,
                      const int* outn, const int* outl) {
    const int n = *outn;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p = outl[i];
        int lo = 0, hi = nboxes - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pbase[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        outsider_body<P, R>(boxes[lo], p);
    }
}

// ---------------------------------------------------------------------------
// split API: gather+push with global loads; Esirkepov with global atomics
// ---------------------------------------------------------------------------
template <int P, typename R>
__global__ void __launch_bounds__(kBlock) k_gather_push(StepArgs<R> A) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= A.np) return;
    const Geom& g = A.g;
    int cell[3];
    R f0[3];
    double xg0[3] = {0.0, 0.0, 0.0};
    if (sizeof(R) == 8) {
        for (int a = 0; a < 3; ++a) {
            xg0[a] = double(A.pa[a][p]);
            double f;
            split_pos(xg0[a], g.d[a], g.n[a], cell[a], f);
            f0[a] = R(f);
        }
    } else {
        cell_of(g, A.key[p], cell[0], cell[1], cell[2]);
        for (int a = 0; a < 3; ++a) f0[a] = A.pa[a][p];
    }
    R u[3] = {A.pa[3][p], A.pa[4][p], A.pa[5][p]};
    GatherW<P, R> G;
    int fn[3], fs[3];
    gather_weights<P, R>(f0, G, fn, fs);
    offsets_global<P, R>(G, g, cell, fn, fs);
    R EB[6];
    gather6<P, R>(G, A.E, A.B, EB);
    Moved<R> mv;
    push_particle<P, R>(A, EB, cell, f0, xg0, u, mv);
    if (!mv.ok) {
        raise_error(A.err, ERRBIT_PARTICLE);
        // keep the particle where it was; the deposit sees no move
        for (int a = 0; a < 3; ++a) {
            A.old[a][p] = sizeof(R) == 8 ? R(xg0[a]) : f0[a];
            A.old[3 + a][p] = R(0);
        }
        if (sizeof(R) == 4) A.oldkey[p] = A.key[p];
        return;
    }
    for (int a = 0; a < 3; ++a) A.pa[3 + a][p] = mv.u[a];
    int nc[3];
    if (sizeof(R) == 8) {
        for (int a = 0; a < 3; ++a) {
            A.old[a][p] = R(xg0[a]);
            A.old[3 + a][p] = R(mv.xg1[a] - xg0[a]);  // exact: the unwrapped move
            const double xw = wrap_pos(mv.xg1[a], g.L[a]);
            A.pa[a][p] = R(xw);
            double f;
            split_pos(xw, g.d[a], g.n[a], nc[a], f);
        }
    } else {
        A.oldkey[p] = A.key[p];
        for (int a = 0; a < 3; ++a) {
            A.old[a][p] = f0[a];
            A.old[3 + a][p] = mv.f1[a] - f0[a];
            float nf;
            renormalise(float(mv.f1[a]), cell[a], g.n[a], nc[a], nf);
            A.pa[a][p] = R(nf);
        }
    }
    A.key[p] = key_of(g, nc[0], nc[1], nc[2]);
}

template <int P, typename R>
__global__ void __launch_bounds__(kBlock) k_deposit(StepArgs<R> A) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= A.np) return;
    const Geom& g = A.g;
    int cell[3];
    R f0[3], f1[3];
    if (sizeof(R) == 8) {
        for (int a = 0; a < 3; ++a) {
            const double x0 = double(A.old[a][p]);
            double f;
            split_pos(x0, g.d[a], g.n[a], cell[a], f);
            const double x1 = __dadd_rn(x0, double(A.old[3 + a][p]));
            f0[a] = R(f);
            f1[a] = R(x1 / g.d[a] - double(cell[a]));
        }
    } else {
        cell_of(g, A.oldkey[p], cell[0], cell[1], cell[2]);
        for (int a = 0; a < 3; ++a) {
            f0[a] = A.old[a][p];
            f1[a] = f0[a] + A.old[3 + a][p];
        }
    }
    EsirkAxis<P, R> ax[3];
    for (int a = 0; a < 3; ++a) ax[a].init(f0[a], f1[a]);
    const R wq = A.pa[6][p];
    const R coef[3] = {A.jc[0] * wq, A.jc[1] * wq, A.jc[2] * wq};
    JTarget<P, R> jt;
    jtarget_global<P, R>(jt, g, A.J, cell, ax);
    esirkepov_deposit<P, R>(ax, coef, jt);
}

// ---------------------------------------------------------------------------
// Yee FDTD
// ---------------------------------------------------------------------------

// B <- B - h curl E (forward differences: B sits half a cell above E), at cell c.
template <typename R> __device__ __forceinline__ void yee_b_at(const YeeArgs<R>& Y, const int64_t c) {
    const int k = int(c % Y.n[2]);
    const int j = int((c / Y.n[2]) % Y.n[1]);
    const int i = int(c / ((int64_t)Y.n[1] * Y.n[2]));
    const int64_t sx = (int64_t)Y.n[1] * Y.n[2], sy = Y.n[2];
    const int64_t ip = c + (i + 1 == Y.n[0] ? -(int64_t)(Y.n[0] - 1) * sx : sx);
    const int64_t jp = c + (j + 1 == Y.n[1] ? -(int64_t)(Y.n[1] - 1) * sy : sy);
    const int64_t kp = c + (k + 1 == Y.n[2] ? -(int64_t)(Y.n[2] - 1) : 1);
    const R ex = Y.E[0][c], ey = Y.E[1][c], ez = Y.E[2][c];
    const bool top = Y.zopen && k + 1 == Y.n[2];  // z open: E beyond the end is zero
    const R dEz_dy = (Y.E[2][jp] - ez) * Y.inv[1];
    const R dEy_dz = ((top ? R(0) : Y.E[1][kp]) - ey) * Y.inv[2];
    const R dEx_dz = ((top ? R(0) : Y.E[0][kp]) - ex) * Y.inv[2];
    const R dEz_dx = (Y.E[2][ip] - ez) * Y.inv[0];
    const R dEy_dx = (Y.E[1][ip] - ey) * Y.inv[0];
    const R dEx_dy = (Y.E[0][jp] - ex) * Y.inv[1];
    Y.B[0][c] -= Y.h * (dEz_dy - dEy_dz);
    Y.B[1][c] -= Y.h * (dEx_dz - dEz_dx);
    Y.B[2][c] -= Y.h * (dEy_dx - dEx_dy);
}

// E <- E + dt (curl B - J) (backward differences), at cell c.
template <typename R> __device__ __forceinline__ void yee_e_at(const YeeArgs<R>& Y, const int64_t c) {
    const int k = int(c % Y.n[2]);
    const int j = int((c / Y.n[2]) % Y.n[1]);
    const int i = int(c / ((int64_t)Y.n[1] * Y.n[2]));
    const int64_t sx = (int64_t)Y.n[1] * Y.n[2], sy = Y.n[2];
    const int64_t im = c - (i == 0 ? -(int64_t)(Y.n[0] - 1) * sx : sx);
    const int64_t jm = c - (j == 0 ? -(int64_t)(Y.n[1] - 1) * sy : sy);
    const int64_t km = c - (k == 0 ? -(int64_t)(Y.n[2] - 1) : 1);
    const R bx = Y.B[0][c], by = Y.B[1][c], bz = Y.B[2][c];
    const bool bottom = Y.zopen && k == 0;  // z open: B below the start is zero
    const R dBz_dy = (bz - Y.B[2][jm]) * Y.inv[1];
    const R dBy_dz = (by - (bottom ? R(0) : Y.B[1][km])) * Y.inv[2];
    const R dBx_dz = (bx - (bottom ? R(0) : Y.B[0][km])) * Y.inv[2];
    const R dBz_dx = (bz - Y.B[2][im]) * Y.inv[0];
    const R dBy_dx = (by - Y.B[1][im]) * Y.inv[0];
    const R dBx_dy = (bx - Y.B[0][jm]) * Y.inv[1];
    Y.E[0][c] += Y.h * ((dBz_dy - dBy_dz) - Y.J[0][c]);
    Y.E[1][c] += Y.h * ((dBx_dz - dBz_dx) - Y.J[1][c]);
    Y.E[2][c] += Y.h * ((dBy_dx - dBx_dy) - Y.J[2][c]);
}

template <typename R> __global__ void __launch_bounds__(kBlock) k_yee_b(YeeArgs<R> Y) {
    const int64_t C = (int64_t)Y.n[0] * Y.n[1] * Y.n[2];
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (Y.step && c == 0) *Y.step += 1;
    if (c < C) yee_b_at(Y, c);
}

template <typename R> __global__ void __launch_bounds__(kBlock) k_yee_e(YeeArgs<R> Y) {
    const int64_t C = (int64_t)Y.n[0] * Y.n[1] * Y.n[2];
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < C) yee_e_at(Y, c);
}

// Batch of boxes: block b updates cells [blocks[b].y, blocks[b].y + blocks[b].z)
// of box blocks[b].x (a block never spans two boxes).  `step`, when non-null,
// is advanced once.
template <typename R>
__global__ void __launch_bounds__(kBlock)
    k_yee_b_batch(const YeeArgs<R>* __restrict__ boxes, const int4* __restrict__ blocks, long long* step) {
    const int4 bk = blocks[blockIdx.x];
    if (step && blockIdx.x == 0 && threadIdx.x == 0) *step += 1;
    if (int(threadIdx.x) < bk.z) yee_b_at(boxes[bk.x], int64_t(bk.y) + threadIdx.x);
}

template <typename R>
__global__ void __launch_bounds__(kBlock) k_yee_e_batch(const YeeArgs<R>* __restrict__ boxes, const int4* __restrict__ blocks) {
    const int4 bk = blocks[blockIdx.x];
    if (int(threadIdx.x) < bk.z) yee_e_at(boxes[bk.x], int64_t(bk.y) + threadIdx.x);
}

template <typename R> YeeArgs<R> make_yee(pic_ctx* c, double h) {
    YeeArgs<R> Y;
    for (int d = 0; d < 3; ++d) {
        Y.E[d] = static_cast<R*>(c->F[d]);
        Y.B[d] = static_cast<R*>(c->F[3 + d]);
        Y.J[d] = static_cast<const R*>(c->F[6 + d]);
        Y.n[d] = c->g.n[d];
        Y.inv[d] = R(1.0 / c->g.d[d]);
    }
    Y.h = R(h);
    Y.step = nullptr;
    Y.zopen = c->g.zopen;
    return Y;
}

// ---------------------------------------------------------------------------
// particle load / store, field conversion, diagnostics
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_load(StepArgs<R> A, const double* x, const double* y, const double* z, const double* ux,
                       const double* uy, const double* uz, const double* w, int* id, unsigned long long* wmax) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= A.np) return;
    const Geom& g = A.g;
    const double xs[3] = {x[p], y[p], z[p]};
    const double us[3] = {ux[p], uy[p], uz[p]};
    bool ok = isfinite(w[p]);
    int cell[3];
    bool gone = false;  // z open: a particle loaded outside [0, Lz) is dropped by the first sort
    for (int a = 0; a < 3; ++a) {
        ok = ok && isfinite(xs[a]) && isfinite(us[a]);
        double xv = isfinite(xs[a]) ? xs[a] : 0.0;
        if (a == 2 && g.zopen && !(xv >= 0.0 && xv < g.L[2])) gone = true, xv = 0.0;
        xv = fmod(xv, g.L[a]);
        xv = wrap_pos(xv, g.L[a]);
        double f;
        split_pos(xv, g.d[a], g.n[a], cell[a], f);
        if (sizeof(R) == 8) {
            A.pa[a][p] = R(xv);
        } else {
            float ff = float(f);
            if (ff >= 1.0f) {  // rounds up to the next cell
                ff = 0.0f;
                cell[a] = wrap_once(cell[a] + 1, g.n[a]);
            }
            A.pa[a][p] = R(ff);
        }
        A.pa[3 + a][p] = R(us[a]);
    }
    A.pa[6][p] = R(w[p]);
    A.key[p] = gone ? dead_key(g) : key_of(g, cell[0], cell[1], cell[2]);
    id[p] = int(p);
    // largest |w|: non-negative doubles order like their bit patterns
    if (isfinite(w[p])) atomicMax(wmax, (unsigned long long)__double_as_longlong(fabs(double(R(w[p])))));
    if (!ok) raise_error(A.err, ERRBIT_PARTICLE);
}

template <typename R>
__global__ void k_store(StepArgs<R> A, double* x, double* y, double* z, double* ux, double* uy, double* uz,
                        double* w, const int* idsrc, int32_t* id) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= A.np) return;
    const Geom& g = A.g;
    double* xs[3] = {x, y, z};
    double* us[3] = {ux, uy, uz};
    int cell[3];
    if (sizeof(R) == 4) cell_of(g, A.key[p], cell[0], cell[1], cell[2]);
    for (int a = 0; a < 3; ++a) {
        if (xs[a]) {
            double v = sizeof(R) == 8 ? double(A.pa[a][p]) : (double(cell[a]) + double(A.pa[a][p])) * g.d[a];
            xs[a][p] = wrap_pos(v, g.L[a]);
        }
        if (us[a]) us[a][p] = double(A.pa[3 + a][p]);
    }
    if (w) w[p] = double(A.pa[6][p]);
    if (id) id[p] = idsrc[p];
}

template <typename S, typename D> __global__ void k_convert(const S* src, D* dst, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = D(src[i]);
}

// out[0] += sum |F|^2 / 2 over Ex..Bz (times dV on the host), out[1] kinetic,
// out[2] charge, out[3] max |div B| (as a bit pattern, max via atomicMax).
template <typename R>
__global__ void k_diag_fields(const R* const* F, int64_t C, double* out) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < C; i += (int64_t)gridDim.x * blockDim.x)
        for (int c = 0; c < 6; ++c) {
            const double v = double(F[c][i]);
            s += v * v;
        }
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double red[kBlock / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(out, 0.5 * t);
    }
}

template <typename R>
__global__ void k_diag_particles(StepArgs<R> A, double m, double q, double* out) {
    double ke = 0.0, ch = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < A.np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double u0 = A.pa[3][p], u1 = A.pa[4][p], u2 = A.pa[5][p], w = A.pa[6][p];
        ke += w * m * (sqrt(1.0 + u0 * u0 + u1 * u1 + u2 * u2) - 1.0);
        ch += q * w;
    }
    for (int o = 16; o; o >>= 1) {
        ke += __shfl_down_sync(0xffffffffu, ke, o);
        ch += __shfl_down_sync(0xffffffffu, ch, o);
    }
    __shared__ double red[2][kBlock / 32];
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = ke;
        red[1][threadIdx.x >> 5] = ch;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[0][w], b += red[1][w];
        atomicAdd(out + 1, a);
        atomicAdd(out + 2, b);
    }
}

template <typename R>
__global__ void k_diag_divb(const R* Bx, const R* By, const R* Bz, int nx, int ny, int nz, double dx, double dy,
                            double dz, int zopen, unsigned long long* out) {
    const int64_t C = (int64_t)nx * ny * nz;
    double mx = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const int k = int(c % nz), j = int((c / nz) % ny), i = int(c / ((int64_t)ny * nz));
        const int64_t ip = ((int64_t)wrap_once(i + 1, nx) * ny + j) * nz + k;
        const int64_t jp = ((int64_t)i * ny + wrap_once(j + 1, ny)) * nz + k;
        const int64_t kp = ((int64_t)i * ny + j) * nz + wrap_once(k + 1, nz);
        const double bz_up = zopen && k + 1 == nz ? 0.0 : double(Bz[kp]);  // z open: zero beyond the end
        const double v = (double(Bx[ip]) - double(Bx[c])) / dx + (double(By[jp]) - double(By[c])) / dy +
                         (bz_up - double(Bz[c])) / dz;
        mx = fmax(mx, fabs(v));
    }
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// ---------------------------------------------------------------------------
// moving window (z open)
// ---------------------------------------------------------------------------
// F(i,j,k) <- F(i,j,k+1), F(i,j,nz-1) <- 0 in place: one warp per z column
// walks it in chunks of 32 (each element is read before it is overwritten:
// in the same chunk by the warp's load, or by the previous chunk's).
template <typename R>
__global__ void __launch_bounds__(kBlock) k_shift_fields(R* F0, int64_t C, int nz, int64_t columns) {
    const int64_t col = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (col >= columns) return;
    R* f = F0 + (int64_t)blockIdx.y * C + col * nz;
    for (int k0 = 0; k0 < nz; k0 += 32) {
        const int k = k0 + lane;
        const R v = k + 1 < nz ? f[k + 1] : R(0);
        __syncwarp();
        if (k < nz) f[k] = v;
        __syncwarp();
    }
}

// Particles move down one cell along z; those below z = 0 get the removed key.
template <typename R> __global__ void __launch_bounds__(kBlock) k_shift_particles(StepArgs<R> A) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= A.np) return;
    const Geom& g = A.g;
    const int dead = dead_key(g);
    const int key = A.key[p];
    if (key == dead) return;
    int i, j, k;
    if (sizeof(R) == 8) {
        const double z = double(A.pa[2][p]) - g.d[2];
        A.pa[2][p] = R(z);
        if (!(z >= 0.0)) {
            A.key[p] = dead;
            return;
        }
        double f;
        split_pos(double(A.pa[0][p]), g.d[0], g.n[0], i, f);
        split_pos(double(A.pa[1][p]), g.d[1], g.n[1], j, f);
        split_pos(z, g.d[2], g.n[2], k, f);
    } else {
        cell_of(g, key, i, j, k);
        k -= 1;  // the in-cell offset is unchanged
        if (k < 0) {
            A.key[p] = dead;
            return;
        }
    }
    A.key[p] = key_of(g, i, j, k);
}

struct InjectArgs {
    int64_t first;     // first slot (particle index) written
    int64_t first_id;  // id of slot `first`
    int ppc;
    double n0, ramp_start, ramp_length;
    double zlab0;      // lab-frame z of the front slab's lower face
};

// The front slab k = nz-1: in each cell particles m = 0..ppc-1 at in-cell
// offset (m + 1/2)/ppc on every axis, at rest, weight density(lab z) dV / ppc
// with the density rising linearly from 0 at ramp_start over ramp_length to
// n0; where the density is zero the slot gets the removed key.  Slot and id
// follow (i ny + j) ppc + m.
template <typename R> __global__ void __launch_bounds__(kBlock) k_inject(StepArgs<R> A, InjectArgs I, int* id) {
    const Geom& g = A.g;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)g.n[0] * g.n[1] * I.ppc;
    if (t >= total) return;
    const int m = int(t % I.ppc);
    const int64_t ij = t / I.ppc;
    const int j = int(ij % g.n[1]), i = int(ij / g.n[1]);
    const int k = g.n[2] - 1;
    const double off = (m + 0.5) / I.ppc;
    const double zl = I.zlab0 + off * g.d[2];
    double dens;
    if (I.ramp_length > 0.0) dens = I.n0 * fmin(fmax((zl - I.ramp_start) / I.ramp_length, 0.0), 1.0);
    else dens = zl >= I.ramp_start ? I.n0 : 0.0;
    const int64_t p = I.first + t;
    if (sizeof(R) == 8) {
        A.pa[0][p] = R((i + off) * g.d[0]);
        A.pa[1][p] = R((j + off) * g.d[1]);
        A.pa[2][p] = R((k + off) * g.d[2]);
    } else {
        A.pa[0][p] = R(off);
        A.pa[1][p] = R(off);
        A.pa[2][p] = R(off);
    }
    A.pa[3][p] = R(0);
    A.pa[4][p] = R(0);
    A.pa[5][p] = R(0);
    A.pa[6][p] = R(dens * g.d[0] * g.d[1] * g.d[2] / I.ppc);
    A.key[p] = dens > 0.0 ? key_of(g, i, j, k) : dead_key(g);
    id[p] = int(I.first_id + t);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(int64_t n) { return unsigned((n + kBlock - 1) / kBlock); }

template <typename R, int P, class LY> cudaError_t tile_step_impl(pic_ctx* c) {
    StepArgs<R> A = make_args<R>(c);
    const size_t smem = LY::template smem_bytes<R>();
    static size_t configured = 0;  // per instantiation; set outside stream capture by pic_init_grid
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_step<P, R, LY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem));
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    k_tile_step<P, R, LY><<<unsigned(c->g.ntiles), tile_block<R>(), smem, c->stream>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_outsiders<P, R><<<152 * 4, kBlock, 0, c->stream>>>(A);
    return cudaGetLastError();
}

template <typename R, class LY> cudaError_t tile_step_order(pic_ctx* c) {
    switch (c->order) {
    case 1: return tile_step_impl<R, 1, LY>(c);
    case 2: return tile_step_impl<R, 2, LY>(c);
    default: return tile_step_impl<R, 3, LY>(c);
    }
}

template <typename R> cudaError_t tile_step_dispatch(pic_ctx* c) {
    return c->layout == 1 ? tile_step_order<R, LayoutRow<R>>(c) : tile_step_order<R, LayoutCube>(c);
}

cudaError_t launch_tile_step(pic_ctx* c) {
    // J is one allocation of three components (see pic_api.cu); the outsider
    // counter sits after the four error words
    cudaError_t e = cudaMemsetAsync(c->F[6], 0, 3 * c->g.C * c->rsize, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err + 4, 0, sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return e;
    return c->prec == PIC_FP64 ? tile_step_dispatch<double>(c) : tile_step_dispatch<float>(c);
}

// The tile kernels need more than 48 KB of dynamic shared memory: raise the
// limit once, before any stream capture.
cudaError_t configure_tile_kernels(pic_ctx* c) {
    auto set = [](auto kernel, size_t bytes) {
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    };
    cudaError_t e = cudaSuccess;
#define PIC_CFG(R, P, LY)                                                              \
    if (e == cudaSuccess) e = set(k_tile_step<P, R, LY>, LY::template smem_bytes<R>());
    PIC_CFG(float, 1, LayoutRow<float>) PIC_CFG(float, 2, LayoutRow<float>) PIC_CFG(float, 3, LayoutRow<float>)
    PIC_CFG(float, 1, LayoutCube) PIC_CFG(float, 2, LayoutCube) PIC_CFG(float, 3, LayoutCube)
    PIC_CFG(double, 1, LayoutRow<double>) PIC_CFG(double, 2, LayoutRow<double>) PIC_CFG(double, 3, LayoutRow<double>)
    PIC_CFG(double, 1, LayoutCube) PIC_CFG(double, 2, LayoutCube) PIC_CFG(double, 3, LayoutCube)
#undef PIC_CFG
    (void)c;
    return e;
}

// ---- batch of boxes ----------------------------------------------------------
template <typename R, int P> cudaError_t tile_batch_impl(const BatchTileLaunch& L, cudaStream_t s) {
    using LY = LayoutCube;
    if (L.nitems <= 0) return cudaSuccess;
    const size_t smem = LY::template smem_bytes<R>();
    const int grid = L.grid < L.nitems ? L.grid : L.nitems;
    k_tile_step_batch<P, R, LY><<<unsigned(grid), tile_block<R>(), smem, s>>>(
        static_cast<const StepArgs<R>*>(L.boxes), L.items, L.nitems, L.queue);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_outsiders_batch<P, R><<<152 * 2, kBlock, 0, s>>>(static_cast<const StepArgs<R>*>(L.boxes), L.pbase, L.nboxes,
                                                        L.outn, L.outl);
    return cudaGetLastError();
}

cudaError_t launch_tile_step_batch(int prec, const BatchTileLaunch& L, cudaStream_t s) {
    if (prec == PIC_FP64) {
        switch (L.order) {
        case 1: return tile_batch_impl<double, 1>(L, s);
        case 2: return tile_batch_impl<double, 2>(L, s);
        default: return tile_batch_impl<double, 3>(L, s);
        }
    }
    switch (L.order) {
    case 1: return tile_batch_impl<float, 1>(L, s);
    case 2: return tile_batch_impl<float, 2>(L, s);
    default: return tile_batch_impl<float, 3>(L, s);
    }
}

template <typename R>
cudaError_t yee_batch_impl(const void* yb, const void* ye, const int4* blocks, int nblocks, long long* step,
                           cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    const auto* B = static_cast<const YeeArgs<R>*>(yb);
    const auto* E = static_cast<const YeeArgs<R>*>(ye);
    k_yee_b_batch<R><<<unsigned(nblocks), kBlock, 0, s>>>(B, blocks, nullptr);
    k_yee_e_batch<R><<<unsigned(nblocks), kBlock, 0, s>>>(E, blocks);
    k_yee_b_batch<R><<<unsigned(nblocks), kBlock, 0, s>>>(B, blocks, step);
    return cudaGetLastError();
}

cudaError_t launch_yee_batch(int prec, const void* yb, const void* ye, const int4* blocks, int nblocks,
                             long long* step, cudaStream_t s) {
    return prec == PIC_FP64 ? yee_batch_impl<double>(yb, ye, blocks, nblocks, step, s)
                            : yee_batch_impl<float>(yb, ye, blocks, nblocks, step, s);
}

__global__ void k_rekey(int* key, int64_t n, Geom from, Geom to) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int i, j, k;
    cell_of(from, key[p], i, j, k);
    key[p] = key_of(to, i, j, k);
}

cudaError_t launch_rekey(int* key, int64_t n, const Geom& from, const Geom& to, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_rekey<<<blocks_for(n), kBlock, 0, s>>>(key, n, from, to);
    return cudaGetLastError();
}

cudaError_t configure_batch_kernels() {
    auto set = [](auto kernel, size_t bytes) {
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    };
    using LY = LayoutCube;
    cudaError_t e = cudaSuccess;
#define PIC_CFG(R, P) \
    if (e == cudaSuccess) e = set(k_tile_step_batch<P, R, LY>, LY::template smem_bytes<R>());
    PIC_CFG(float, 1) PIC_CFG(float, 2) PIC_CFG(float, 3) PIC_CFG(double, 1) PIC_CFG(double, 2) PIC_CFG(double, 3)
#undef PIC_CFG
    return e;
}

template <typename R, int P> cudaError_t gp_impl(pic_ctx* c) {
    StepArgs<R> A = make_args<R>(c);
    if (c->np == 0) return cudaSuccess;
    k_gather_push<P, R><<<blocks_for(c->np), kBlock, 0, c->stream>>>(A);
    return cudaGetLastError();
}

template <typename R, int P> cudaError_t dep_impl(pic_ctx* c) {
    StepArgs<R> A = make_args<R>(c);
    if (c->np == 0) return cudaSuccess;
    k_deposit<P, R><<<blocks_for(c->np), kBlock, 0, c->stream>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_gather_push_global(pic_ctx* c) {
    if (c->prec == PIC_FP64) {
        switch (c->order) {
        case 1: return gp_impl<double, 1>(c);
        case 2: return gp_impl<double, 2>(c);
        default: return gp_impl<double, 3>(c);
        }
    }
    switch (c->order) {
    case 1: return gp_impl<float, 1>(c);
    case 2: return gp_impl<float, 2>(c);
    default: return gp_impl<float, 3>(c);
    }
}

cudaError_t launch_deposit_global(pic_ctx* c) {
    cudaError_t e = cudaMemsetAsync(c->F[6], 0, 3 * c->g.C * c->rsize, c->stream);
    if (e != cudaSuccess) return e;
    if (c->prec == PIC_FP64) {
        switch (c->order) {
        case 1: return dep_impl<double, 1>(c);
        case 2: return dep_impl<double, 2>(c);
        default: return dep_impl<double, 3>(c);
        }
    }
    switch (c->order) {
    case 1: return dep_impl<float, 1>(c);
    case 2: return dep_impl<float, 2>(c);
    default: return dep_impl<float, 3>(c);
    }
}

cudaError_t launch_yee_b(pic_ctx* c, double h) {
    if (c->prec == PIC_FP64) {
        auto Y = make_yee<double>(c, h);
        k_yee_b<double><<<blocks_for(c->g.C), kBlock, 0, c->stream>>>(Y);
    } else {
        auto Y = make_yee<float>(c, h);
        k_yee_b<float><<<blocks_for(c->g.C), kBlock, 0, c->stream>>>(Y);
    }
    return cudaGetLastError();
}

cudaError_t launch_yee_e(pic_ctx* c) {
    if (c->prec == PIC_FP64) {
        auto Y = make_yee<double>(c, c->dt);
        k_yee_e<double><<<blocks_for(c->g.C), kBlock, 0, c->stream>>>(Y);
    } else {
        auto Y = make_yee<float>(c, c->dt);
        k_yee_e<float><<<blocks_for(c->g.C), kBlock, 0, c->stream>>>(Y);
    }
    return cudaGetLastError();
}

__global__ void k_step_counter(long long* s) { *s += 1; }

cudaError_t launch_step_counter(pic_ctx* c) {
    k_step_counter<<<1, 1, 0, c->stream>>>(c->d_step);
    return cudaGetLastError();
}

cudaError_t launch_load_particles(pic_ctx* c, const double* const src[7], int64_t n) {
    if (n == 0) return cudaSuccess;
    if (c->prec == PIC_FP64) {
        auto A = make_args<double>(c);
        k_load<double><<<blocks_for(n), kBlock, 0, c->stream>>>(A, src[0], src[1], src[2], src[3], src[4], src[5],
                                                               src[6], c->P[c->cur].id,
                                                               reinterpret_cast<unsigned long long*>(c->err + 6));
    } else {
        auto A = make_args<float>(c);
        k_load<float><<<blocks_for(n), kBlock, 0, c->stream>>>(A, src[0], src[1], src[2], src[3], src[4], src[5],
                                                              src[6], c->P[c->cur].id,
                                                              reinterpret_cast<unsigned long long*>(c->err + 6));
    }
    return cudaGetLastError();
}

cudaError_t launch_get_particles(pic_ctx* c, double* const dst[7], int32_t* id) {
    if (c->np == 0) return cudaSuccess;
    if (c->prec == PIC_FP64) {
        auto A = make_args<double>(c);
        k_store<double><<<blocks_for(c->np), kBlock, 0, c->stream>>>(A, dst[0], dst[1], dst[2], dst[3], dst[4],
                                                                    dst[5], dst[6], c->P[c->cur].id, id);
    } else {
        auto A = make_args<float>(c);
        k_store<float><<<blocks_for(c->np), kBlock, 0, c->stream>>>(A, dst[0], dst[1], dst[2], dst[3], dst[4],
                                                                   dst[5], dst[6], c->P[c->cur].id, id);
    }
    return cudaGetLastError();
}

cudaError_t launch_field_to_f64(pic_ctx* c, int which, double* dst) {
    if (c->prec == PIC_FP64)
        return cudaMemcpyAsync(dst, c->F[which], c->g.C * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    k_convert<float, double><<<blocks_for(c->g.C), kBlock, 0, c->stream>>>(static_cast<const float*>(c->F[which]),
                                                                         dst, c->g.C);
    return cudaGetLastError();
}

cudaError_t launch_field_from_f64(pic_ctx* c, int which, const double* src) {
    if (c->prec == PIC_FP64)
        return cudaMemcpyAsync(c->F[which], src, c->g.C * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    k_convert<double, float><<<blocks_for(c->g.C), kBlock, 0, c->stream>>>(src, static_cast<float*>(c->F[which]),
                                                                         c->g.C);
    return cudaGetLastError();
}

template <typename R> cudaError_t diag_impl(pic_ctx* c, double* d_out) {
    // F pointer table lives in the scratch after the four outputs
    const R** tab = reinterpret_cast<const R**>(d_out + 8);
    const R* host_tab[6];
    for (int i = 0; i < 6; ++i) host_tab[i] = static_cast<const R*>(c->F[i]);
    cudaError_t e = cudaMemcpyAsync(tab, host_tab, sizeof(host_tab), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return e;
    const unsigned nb = 152 * 4;
    k_diag_fields<R><<<nb, kBlock, 0, c->stream>>>(tab, c->g.C, d_out);
    if (c->np > 0) {
        auto A = make_args<R>(c);
        k_diag_particles<R><<<nb, kBlock, 0, c->stream>>>(A, c->m, c->q, d_out);
    }
    k_diag_divb<R><<<nb, kBlock, 0, c->stream>>>(static_cast<const R*>(c->F[3]), static_cast<const R*>(c->F[4]),
                                                 static_cast<const R*>(c->F[5]), c->g.n[0], c->g.n[1], c->g.n[2],
                                                 c->g.d[0], c->g.d[1], c->g.d[2], c->g.zopen,
                                                 reinterpret_cast<unsigned long long*>(d_out + 3));
    return cudaGetLastError();
}

cudaError_t launch_diagnostics(pic_ctx* c, double* d_out) {
    return c->prec == PIC_FP64 ? diag_impl<double>(c, d_out) : diag_impl<float>(c, d_out);
}

template <typename R> cudaError_t window_shift_impl(pic_ctx* c) {
    const int64_t columns = int64_t(c->g.n[0]) * c->g.n[1];
    const dim3 grid(unsigned((columns * 32 + kBlock - 1) / kBlock), 9);
    k_shift_fields<R><<<grid, kBlock, 0, c->stream>>>(static_cast<R*>(c->F[0]), c->g.C, c->g.n[2], columns);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || c->np == 0) return e;
    k_shift_particles<R><<<blocks_for(c->np), kBlock, 0, c->stream>>>(make_args<R>(c));
    return cudaGetLastError();
}

cudaError_t launch_window_shift(pic_ctx* c) {
    return c->prec == PIC_FP64 ? window_shift_impl<double>(c) : window_shift_impl<float>(c);
}

template <typename R> cudaError_t inject_impl(pic_ctx* c) {
    InjectArgs I;
    I.first = c->np;
    I.first_id = c->next_id;
    I.ppc = c->inj_ppc;
    I.n0 = c->inj_n0;
    I.ramp_start = c->inj_ramp_start;
    I.ramp_length = c->inj_ramp_length;
    I.zlab0 = double(c->shifts + c->g.n[2] - 1) * c->g.d[2];
    const int64_t total = int64_t(c->g.n[0]) * c->g.n[1] * c->inj_ppc;
    if (total == 0) return cudaSuccess;
    k_inject<R><<<blocks_for(total), kBlock, 0, c->stream>>>(make_args<R>(c), I, c->P[c->cur].id);
    return cudaGetLastError();
}

cudaError_t launch_inject(pic_ctx* c) {
    return c->prec == PIC_FP64 ? inject_impl<double>(c) : inject_impl<float>(c);
}

}  // namespace pic
