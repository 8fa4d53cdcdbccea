// Particle kernels of libpic (sm_103a).
//
//  k_tile_step        fused gather + Boris + advance + Esirkepov for one tile
//                     of cells per CTA: E/B of the tile and its halo staged in
//                     shared memory, J accumulated in shared memory, one
//                     vectorised atomic flush per tile (Sec. 3.1 fuses gather
//                     and push; Sec. 3.4 discusses shared-memory buffers).
//  k_tile_step_batch  the same tile body for (box, tile) items of a batch of
//                     boxes, pulled from a queue by a persistent grid.
//  k_outsiders        particles outside their tile (between sorts): global
//                     gather and global atomics.
//  k_gather_push      one particle per thread, fields read from global memory.
//  k_deposit          one particle per thread, Esirkepov with global atomics
//                     (the paper's GPU deposit, Sec. 3.4.1).
// The Yee update, load/store, diagnostics and the moving window are in
// pic_support.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
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
// take the particles of one z-row of 32 cells (tile_body), and with row and
// plane pitches that are multiples of 32 words the bank of every access is
// its z index, so lanes in distinct cells hit distinct banks whatever their
// staggering offsets along x and y.  Otherwise up to 8 x 8 x 8 cells.
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
using LayoutRow = std::conditional_t<sizeof(R) == 4, Layout<4, 4, 32, 64, 64>, Layout<4, 4, 32, 38, 40>>;
// 8x8x8 tiles: the 32 cells of a warp are 4 z-rows of 8; FP32-mixed row
// pitches of 24 words put those rows on banks 0, 24, 16 and 8 (mod 32), so
// rows never share a bank at the same z.  FP64 keeps compact pitches.
template <typename R>
using LayoutCube = std::conditional_t<sizeof(R) == 4, Layout<8, 8, 8, 24, 24>, Layout<8, 8, 8, 14, 20>>;

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
// (< 1 cell), and Q <= 1.  vscale is the largest power of two with
// vscale max|coef| <= 2^30, so x = rn(v vscale) fits in 31 bits, and because
// scaling by a power of two is exact, vscale is folded into the particle's
// coefficient.  Two int32 arrays take, by native shared-memory integer
// reductions, H = sum (x >> 15) and W = sum x modulo 2^32.  With at most 65535
// particles per tile H cannot overflow (65535 * 2^15 < 2^31), and the low
// part L = sum (x & 0x7fff) = sum x - 2^15 H lies in [0, 65535 * 32767], below
// 2^31, so W - 2^15 H taken modulo 2^32 is L exactly.  The sums are exact and
// independent of order; the flush rebuilds H 2^15 + L.
__device__ __forceinline__ void red_fixed(int* w, int* hi, float v_scaled) {
    const int x = __float2int_rn(v_scaled);
    atomicAdd(w, x);
    atomicAdd(hi, x >> 15);
}

// The low part L of a node from its two sums (see red_fixed).
__device__ __forceinline__ int fixed_low(int hi, int w) { return int(unsigned(w) - (unsigned(hi) << 15)); }

template <int P, class LY, int NC = P + 1, int NT = P + 2>
__device__ __forceinline__ void esirkepov_smem_fixed(int* __restrict__ sJ, int base, const EsirkAxis<P, float> ax[3],
                                                     const float coef_in[3], float vscale) {
    const float coef[3] = {coef_in[0] * vscale, coef_in[1] * vscale, coef_in[2] * vscale};  // exact: power of two
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
                    red_fixed(jx + o, jx + H + o, cum[i] * Q);
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
                    red_fixed(jy + o, jy + H + o, cum[j] * Q);
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
                    red_fixed(jz + o, jz + H + o, cum[kk] * Q);
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

// A fixed-point node sum hi 2^15 + lo (|hi| < 2^31, 0 <= lo < 2^31, as the
// deposit accumulates them) rounded once to float, in FP32 arithmetic: with
// the carry of lo moved into hi both parts are exact floats, and one fused
// multiply-add rounds the exact sum.  Sums of 2^38 and more take the 64-bit
// conversion.
__device__ __forceinline__ float fixed_to_float(int hi, int lo) {
    if (hi > -(1 << 23) && hi < (1 << 23)) return fmaf(float(hi + (lo >> 15)), 32768.0f, float(lo & 0x7fff));
    return __ll2float_rn((long long)hi * 32768 + lo);
}

// Block size of the tile kernel: FP32-mixed 512 threads (one CTA per SM, its
// shared memory holding the fixed-point J box), FP64 256.
template <typename R> constexpr int tile_block() { return sizeof(R) == 4 ? 512 : 256; }

// Periodic index of a cell at most one period outside [0, n) (any i, n > 0,
// without a division in that common case).
__device__ __forceinline__ int wrap_near(int i, int n) {
    if (i < 0) i += n;
    else if (i >= n) i -= n;
    return unsigned(i) < unsigned(n) ? i : wrap_any(i, n);
}

// Stage the sub-box [a0,a1) x [b0,b1) x [k0,k1) of the tile's E/B block (cells
// [-2, T+2) per axis around the tile origin oi, oj, ok), periodic wrap in x, y
// and in z unless z is open, where nothing lies beyond the ends.
// kFull: the whole block of the layout's own tile shape (compile-time
// divisors; the sub-box arguments are ignored).
template <typename R, class LY, bool kFull = false>
__device__ __forceinline__ void stage_box(const StepArgs<R>& A, R* sEB, int oi, int oj, int ok, int a0, int a1, int b0,
                                          int b1, int k0, int k1) {
    const Geom& g = A.g;
    if (kFull) a0 = 0, b0 = 0, k0 = 0;
    const int eb = kFull ? LY::EY : b1 - b0, ek = kFull ? LY::EZ : k1 - k0;
    const int vol = kFull ? LY::EX * LY::EY * LY::EZ : (a1 - a0) * eb * ek;
    for (int e = threadIdx.x; e < 6 * vol; e += blockDim.x) {
        const int c = e / vol;
        int r = e - c * vol;
        const int a = a0 + r / (eb * ek);
        r -= (a - a0) * eb * ek;
        const int b = b0 + r / ek;
        const int kk = k0 + r - (b - b0) * ek;
        const int gi = wrap_near(oi - 2 + a, g.n[0]);
        const int gj = wrap_near(oj - 2 + b, g.n[1]);
        const int kz = ok - 2 + kk;
        R v = R(0);
        if (!g.zopen || unsigned(kz) < unsigned(g.n[2])) {
            const int gk = wrap_near(kz, g.n[2]);
            const int64_t gidx = ((int64_t)gi * g.n[1] + gj) * g.n[2] + gk;
            PIC_CHECK_OR(gidx >= 0 && gidx < g.C && a < LY::EX && b < LY::EY && kk < LY::EZ, A.err, 2, gidx,
                         continue);
            v = c < 3 ? A.E[c][gidx] : A.B[c - 3][gidx];
        }
        sEB[c * LY::eVol + a * LY::eX + b * LY::eY + kk] = v;
    }
}

// TMA staging: one 4-D box (z, y, x, component) of eY x EY x EX x 6 values
// lands in the E/B block exactly (eY, the row pitch, spans a multiple of 16
// bytes and at least EZ + 2 values).  The box starts at z = ok - 4 (TMA wants
// the innermost coordinate on a 16-byte boundary), so the block is addressed
// 2 values in; coordinates outside the grid read
// as zero and the wrapped halo planes are restaged by stage_box after the
// copy has landed.
constexpr int kTmaSpinLimit = 1 << 20;

template <class LY, typename R> __host__ __device__ constexpr bool tma_layout() {
    return (LY::eY * sizeof(R)) % 16 == 0 && LY::EZ + 2 <= LY::eY && LY::eY <= 256;
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
    const unsigned b = unsigned(__cvta_generic_to_shared(bar));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
    const unsigned b = unsigned(__cvta_generic_to_shared(bar));
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(b) : "memory");
}

// Issued by one thread.  The proxy fence orders this CTA's earlier generic
// accesses to the block (a previous tile's loads and stores) before the copy.
__device__ __forceinline__ void tma_load_eb(const CUtensorMap* map, void* dst, unsigned long long* bar, unsigned bytes,
                                            int z, int y, int x) {
    const unsigned d = unsigned(__cvta_generic_to_shared(dst));
    const unsigned b = unsigned(__cvta_generic_to_shared(bar));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(d),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(z), "r"(y), "r"(x), "r"(0), "r"(b)
        : "memory");
}

// Bounded wait for phase `parity` of the barrier; false if it did not complete.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int limit) {
    const unsigned b = unsigned(__cvta_generic_to_shared(bar));
    for (int i = 0; i < limit; ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(b), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Flush of the fixed-point J box in groups of 4 consecutive z nodes (aligned
// float4 reductions into HBM).  JYc, Q4c > 0: the box extents are the
// layout's (compile-time divisors); 0: the runtime jy, q4.
template <typename R, class LY, int JYc, int Q4c>
__device__ __forceinline__ void flush_fixed4(const StepArgs<R>& A, const int* sJi, int oi, int oj, int ok, int jx,
                                             int jy_rt, int q4_rt) {
    const Geom& g = A.g;
    const int jy = JYc > 0 ? JYc : jy_rt;
    const int q4 = Q4c > 0 ? Q4c : q4_rt;
    const int per_c = jx * jy * q4;
    for (int e = threadIdx.x; e < 3 * per_c; e += blockDim.x) {
        const int c = e / per_c;
        int r = e - c * per_c;
        const int row = r / q4;
        const int q = r - row * q4;
        const int a = row / jy;
        const int b = row - a * jy;
        const int o = 2 * c * LY::jVol + a * LY::jX + b * LY::jY + 4 * q;
        const int4 lo = *reinterpret_cast<const int4*>(sJi + o);
        const int4 hi = *reinterpret_cast<const int4*>(sJi + o + LY::jVol);
        if ((lo.x | lo.y | lo.z | lo.w | hi.x | hi.y | hi.z | hi.w) == 0) continue;
        // a group of 4 starts at a multiple of 4 and nz % 4 == 0: it is all inside or all beyond the z ends
        if (g.zopen && unsigned(ok - 4 + 4 * q) >= unsigned(g.n[2])) continue;
        const float4 v = make_float4(fixed_to_float(hi.x, fixed_low(hi.x, lo.x)) * A.inv_vscale,
                                     fixed_to_float(hi.y, fixed_low(hi.y, lo.y)) * A.inv_vscale,
                                     fixed_to_float(hi.z, fixed_low(hi.z, lo.z)) * A.inv_vscale,
                                     fixed_to_float(hi.w, fixed_low(hi.w, lo.w)) * A.inv_vscale);
        const int gi = wrap_near(oi - 2 + a, g.n[0]);
        const int gj = wrap_near(oj - 2 + b, g.n[1]);
        const int gk = wrap_near(ok - 4 + 4 * q, g.n[2]);
        PIC_CHECK_OR(gk + 3 < g.n[2] && ((gk & 3) == 0), A.err, 6, gk, continue);
        float* dst = reinterpret_cast<float*>(A.J[c]) + ((int64_t)gi * g.n[1] + gj) * g.n[2] + gk;
        atomicAdd(reinterpret_cast<float4*>(dst), v);
    }
}

// One tile t of the box described by A, by the whole CTA; `smem_raw` is the
// CTA's dynamic shared memory; `tmap` the TMA descriptor of the box's E/B
// (null: staged by loads).  Returns with the block converged.
template <int P, typename R, class LY>
__device__ __forceinline__ void tile_body(const StepArgs<R>& A, const int t, unsigned char* smem_raw,
                                          const CUtensorMap* tmap = nullptr) {
    R* sm = reinterpret_cast<R*>(smem_raw);
    const Geom& g = A.g;
    constexpr bool kFixed = sizeof(R) == 4;
    constexpr bool kTmaLayout = tma_layout<LY, R>();
    constexpr int kZShift = kTmaLayout ? 2 : 0;
    R* sEB = sm + kZShift;        // 6 * eVol (addressed kZShift elements into the block)
    R* sJ = sm + 6 * LY::eVol;    // FP64: 3 * jVol doubles; FP32-mixed: 6 * jVol int32 (lo, hi per component)
    int* sJi = reinterpret_cast<int*>(sJ);

    const int beg = A.offsets[(int64_t)t * g.cpt];
    const int end = A.offsets[(int64_t)(t + 1) * g.cpt];
    if (end <= beg) return;
    PIC_CHECK_OR(beg >= 0 && end <= A.np, A.err, 1, ((long long)beg << 32) | unsigned(end), return);
    int oi, oj, ok;
    tile_origin(g, t, oi, oj, ok);

    // stage E, B of the tile and a halo of 2 (wrapped), zero the tile's J
    __shared__ __align__(8) unsigned long long s_bar;
    bool by_tma = false;
    {
        const int ex = g.T[0] + 4, ey = g.T[1] + 4, ez = g.T[2] + 4;
        if constexpr (kTmaLayout) {
            by_tma = tmap != nullptr && (unsigned(__cvta_generic_to_shared(sm)) & 127u) == 0u &&
                     ((ok - 2 - kZShift) & 3) == 0;
            if (by_tma) {
                if (threadIdx.x == 0) mbar_init(&s_bar);
                __syncthreads();
                if (threadIdx.x == 0)
                    tma_load_eb(tmap, sm, &s_bar, unsigned(6 * LY::eVol * sizeof(R)), ok - 2 - kZShift, oj - 2,
                                oi - 2);
                for (int e = threadIdx.x; e < 6 * LY::jVol / 4; e += blockDim.x)
                    reinterpret_cast<int4*>(sJi)[e] = make_int4(0, 0, 0, 0);
                // every thread waits for the copy; if it did not land in time,
                // all wait once more (it is still writing into this CTA's
                // shared memory) and the tile is skipped with the error set
                const bool late = __syncthreads_or(!mbar_wait(&s_bar, 0u, kTmaSpinLimit));
                if (late) {
                    if (threadIdx.x == 0) raise_error(A.err, ERRBIT_TIMEOUT);
                    mbar_wait(&s_bar, 0u, kTmaSpinLimit);
                    __syncthreads();
                    return;
                }
                // halo planes that wrap around the grid came in as zeros
                if (oi < 2) stage_box<R, LY>(A, sEB, oi, oj, ok, 0, 2 - oi, 0, ey, 0, ez);
                if (oi + ex - 2 > g.n[0]) stage_box<R, LY>(A, sEB, oi, oj, ok, g.n[0] - oi + 2, ex, 0, ey, 0, ez);
                if (oj < 2) stage_box<R, LY>(A, sEB, oi, oj, ok, 0, ex, 0, 2 - oj, 0, ez);
                if (oj + ey - 2 > g.n[1]) stage_box<R, LY>(A, sEB, oi, oj, ok, 0, ex, g.n[1] - oj + 2, ey, 0, ez);
                if (!g.zopen) {
                    if (ok < 2) stage_box<R, LY>(A, sEB, oi, oj, ok, 0, ex, 0, ey, 0, 2 - ok);
                    if (ok + ez - 2 > g.n[2]) stage_box<R, LY>(A, sEB, oi, oj, ok, 0, ex, 0, ey, g.n[2] - ok + 2, ez);
                }
            }
        }
        if (!by_tma) {
            if (ex == LY::EX && ey == LY::EY && ez == LY::EZ)
                stage_box<R, LY, true>(A, sEB, oi, oj, ok, 0, ex, 0, ey, 0, ez);
            else
                stage_box<R, LY>(A, sEB, oi, oj, ok, 0, ex, 0, ey, 0, ez);
            // J box zeroed 16 bytes at a time (jVol is a multiple of 4; the box starts 16-byte aligned)
            const int n16 = kFixed ? 6 * LY::jVol / 4 : 3 * LY::jVol / 2;
            for (int e = threadIdx.x; e < n16; e += blockDim.x) reinterpret_cast<int4*>(sJ)[e] = make_int4(0, 0, 0, 0);
        }
    }
    __syncthreads();
    if (by_tma && threadIdx.x == 0) mbar_inval(&s_bar);  // every thread is past its wait

    // The tile's particles are cell-sorted; consecutive lanes take consecutive
    // runs of them, so the lanes of a warp work in neighbouring cells (distinct
    // shared-memory banks).  When the tile's cells split evenly over the warps
    // and the particles are spread evenly enough (no warp's share above 1.25x
    // the mean + 32), warp w owns the w-th group of cells (one z-row of the
    // FP32-mixed tile) and its lanes split that group's particles: no two
    // warps then deposit into the same row at the same time.  Otherwise the
    // whole tile is cut into runs of about one cell's worth (or A.run).
    const int cnt = end - beg;
    const int lane = threadIdx.x & 31;
    const int nwarp = blockDim.x >> 5;
    int wbeg = beg, wend = end, run, nrun, rstart, rstride;
    bool by_warp = false;
    if (A.run <= 0 && g.cpt % nwarp == 0 && nwarp <= 32) {
        const int cpw = g.cpt / nwarp;
        const int64_t c0 = (int64_t)t * g.cpt;
        const int gsize = lane < nwarp ? A.offsets[c0 + (int64_t)(lane + 1) * cpw] - A.offsets[c0 + (int64_t)lane * cpw] : 0;
        const int gmax = __reduce_max_sync(0xffffffffu, gsize);
        by_warp = int64_t(gmax) * nwarp * 4 <= int64_t(cnt) * 5 + int64_t(128) * nwarp;
        if (by_warp) {
            const int wid = threadIdx.x >> 5;
            wbeg = A.offsets[c0 + (int64_t)wid * cpw];
            wend = A.offsets[c0 + (int64_t)(wid + 1) * cpw];
            PIC_CHECK_OR(beg <= wbeg && wbeg <= wend && wend <= end, A.err, 1,
                         ((long long)wbeg << 32) | unsigned(wend), wbeg = wend = beg);
        }
    }
    if (by_warp) {
        run = max(1, (wend - wbeg + 31) >> 5);
        nrun = (wend - wbeg + run - 1) / run;  // at most 32: one pass of the warp
        rstart = 0;
        rstride = 32;
    } else {
        run = A.run > 0 ? A.run : max(1, (cnt + (g.cpt >> 1)) / g.cpt);
        nrun = (cnt + run - 1) / run;
        rstart = threadIdx.x - lane;
        rstride = blockDim.x;
    }
    // Warps step their lanes' runs in lockstep.  A move whose old and new
    // shapes start on the same node along every axis (most moves: crossing a
    // cell face is rare) deposits the narrow stencil at once; the others go to
    // a per-warp queue held one slot per lane in registers and are deposited
    // 32 at a time with the full window, so neither kind runs with idle lanes.
    TileMove<R> qs = TileMove<R>::zero();  // this lane's queue slot
    int qn = 0;                            // queued moves (warp-uniform)
    for (int rbase = rstart; rbase < nrun; rbase += rstride) {
        const int rr = rbase + lane;
        const int p0 = wbeg + rr * run;
        const int len = rr < nrun ? min(run, wend - p0) : 0;
        const int maxlen = __reduce_max_sync(0xffffffffu, len);
        // the next particle's loads are issued before the current one's work
        RawParticle<R> next;
        if (len > 0) load_raw<R>(A, p0, next);
        for (int it = 0; it < maxlen; ++it) {
            const int p = p0 + it;
            bool wide = false;
            TileMove<R> mine = TileMove<R>::zero();
            const RawParticle<R> raw = next;
            if (it + 1 < len) load_raw<R>(A, p + 1, next);
            if (it < len) {
                int cell[3];
                R f0[3], u[3], wq;
                double xg0[3];
                decode_particle<R>(A, raw, cell, f0, xg0, u, wq);
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
                        gather_weights<P, R>(f0, G, fn, fs, A.egather != 0);
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
        // the layout's own tile shape indexes the J box with constants
        if (jx == LY::JX && jy == LY::JY && jz == LY::JZ)
            flush_fixed4<R, LY, LY::JY, LY::JZ / 4>(A, sJi, oi, oj, ok, jx, jy, jz / 4);
        else
            flush_fixed4<R, LY, 0, 0>(A, sJi, oi, oj, ok, jx, jy, jz / 4);
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
                v = R(fixed_to_float(sJi[2 * c * LY::jVol + LY::jVol + o],
                                     fixed_low(sJi[2 * c * LY::jVol + LY::jVol + o], sJi[2 * c * LY::jVol + o])) *
                      A.inv_vscale);
            else
                v = sJ[c * LY::jVol + o];
            if (v == R(0)) continue;
            if (g.zopen && unsigned(ok - 4 + kk) >= unsigned(g.n[2])) continue;
            const int gi = wrap_near(oi - 2 + a, g.n[0]);
            const int gj = wrap_near(oj - 2 + b, g.n[1]);
            const int gk = wrap_near(ok - 4 + kk, g.n[2]);
            atomicAdd(A.J[c] + ((int64_t)gi * g.n[1] + gj) * g.n[2] + gk, v);
        }
    }
}

template <int P, typename R, class LY>
__global__ void __launch_bounds__(tile_block<R>(), 1)
    k_tile_step(StepArgs<R> A, const __grid_constant__ CUtensorMap tmap, int use_tma) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    tile_body<P, R, LY>(A, int(blockIdx.x), smem_raw, use_tma ? &tmap : nullptr);
}

// Batch of boxes: a persistent grid pulls (box, tile) items from a queue
// counter (zeroed before the launch); each item's box arguments are copied
// into shared memory first.  Items are ordered heaviest first.
template <int P, typename R, class LY>
__global__ void __launch_bounds__(tile_block<R>(), 1)
    k_tile_step_batch(const StepArgs<R>* __restrict__ boxes, const int2* __restrict__ items, int nitems, int* queue) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
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
        tile_body<P, R, LY>(sA, bt.y, smem_raw, sA.tmap);
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
        gather_weights<P, R>(f0, G, fn, fs, A.egather != 0);
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
    gather_weights<P, R>(f0, G, fn, fs, A.egather != 0);
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
    k_tile_step<P, R, LY><<<unsigned(c->g.ntiles), tile_block<R>(), smem, c->stream>>>(A, c->tmap_eb, c->tma ? 1 : 0);
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
    return c->layout == 1 ? tile_step_order<R, LayoutRow<R>>(c) : tile_step_order<R, LayoutCube<R>>(c);
}

cudaError_t launch_tile_step(pic_ctx* c) {
    // J is one allocation of three components (see pic_api.cu); the outsider
    // counter sits after the four error words
    cudaError_t e = cudaMemsetAsync(c->F[6], 0, 3 * c->g.C * c->rsize, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err + 4, 0, sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return e;
    return c->prec == PIC_FP64 ? tile_step_dispatch<double>(c) : tile_step_dispatch<float>(c);
}

bool encode_eb_tensor_map(CUtensorMap* map, const void* base, const int n[3], int64_t comp_stride, int layout,
                          int prec) {
    std::memset(map, 0, sizeof(*map));
    const cuuint64_t rs = prec == PIC_FP64 ? 8 : 4;
    if ((n[2] * rs) % 16 != 0 || (comp_stride * rs) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0)
        return false;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return false;
    }
    const bool f64 = prec == PIC_FP64;
    const cuuint32_t bz = layout == 1 ? (f64 ? LayoutRow<double>::eY : LayoutRow<float>::eY)
                                      : (f64 ? LayoutCube<double>::eY : LayoutCube<float>::eY);
    const cuuint32_t by = layout == 1 ? LayoutRow<float>::EY : LayoutCube<float>::EY;  // same for both precisions
    const cuuint32_t bx = layout == 1 ? LayoutRow<float>::EX : LayoutCube<float>::EX;
    const cuuint64_t nz = cuuint64_t(n[2]), ny = cuuint64_t(n[1]), nx = cuuint64_t(n[0]);
    const cuuint64_t dims[4] = {nz, ny, nx, 6};
    const cuuint64_t strides[3] = {nz * rs, ny * nz * rs, cuuint64_t(comp_stride) * rs};  // bytes, dimensions 1..3
    const cuuint32_t box[4] = {bz, by, bx, 6};
    const cuuint32_t estride[4] = {1, 1, 1, 1};
    const CUresult r = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn)(
        map, f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dims,
        strides, box, estride,
        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

void setup_tile_tma(pic_ctx* c) {
    c->tma = false;
    std::memset(&c->tmap_eb, 0, sizeof(c->tmap_eb));
    c->tma = encode_eb_tensor_map(&c->tmap_eb, c->F[0], c->g.n, c->g.C, c->layout, c->prec);
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
    PIC_CFG(float, 1, LayoutCube<float>) PIC_CFG(float, 2, LayoutCube<float>) PIC_CFG(float, 3, LayoutCube<float>)
    PIC_CFG(double, 1, LayoutRow<double>) PIC_CFG(double, 2, LayoutRow<double>) PIC_CFG(double, 3, LayoutRow<double>)
    PIC_CFG(double, 1, LayoutCube<double>) PIC_CFG(double, 2, LayoutCube<double>) PIC_CFG(double, 3, LayoutCube<double>)
#undef PIC_CFG
    (void)c;
    return e;
}

// ---- batch of boxes ----------------------------------------------------------
template <typename R, int P> cudaError_t tile_batch_impl(const BatchTileLaunch& L, cudaStream_t s) {
    using LY = LayoutCube<R>;
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

cudaError_t configure_batch_kernels() {
    auto set = [](auto kernel, size_t bytes) {
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    };
    cudaError_t e = cudaSuccess;
#define PIC_CFG(R, P) \
    if (e == cudaSuccess) e = set(k_tile_step_batch<P, R, LayoutCube<R>>, LayoutCube<R>::template smem_bytes<R>());
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

}  // namespace pic
