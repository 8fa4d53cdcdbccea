// Particle kernels of libpic (sm_103a).
//
//  k_tile_step        fused gather + Boris + advance + Esirkepov for one tile
//                     of cells per CTA: E/B of the tile and its halo staged in
//                     shared memory, J accumulated in shared memory, one
//                     vectorised atomic flush per tile (Sec. 3.1 fuses gather
//                     and push; Sec. 3.4 discusses shared-memory buffers).
//  k_tile_step_batch  the same pipelined tile loop over (box, tile) items of a
//                     batch of boxes, pulled from a queue by a persistent grid.
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
#include <utility>

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
//   E/B box: cells [-H, T+H) per axis, z rows of pitch EP
//   J box:   x, y [-H, T+H+1), z [-4, T+4), z rows of pitch JP (z padded so the
//            flush moves aligned float4s)
// H is the halo the shape order needs: the gather of order p reaches nodes
// -2..+2 around a particle's cell for p = 2, 3 and -1..+1 for p = 1, and the
// Esirkepov window of a move shorter than a cell one node further up.
// Layouts.  4 x 4 x 32 when nz is a multiple of 32: the lanes of a warp take
// the particles of z-rows of 32 cells, and with row and plane pitches that
// are multiples of 32 words the bank of every access is its z index, so lanes
// in distinct cells hit distinct banks whatever their staggering offsets
// along x and y.  Otherwise up to 8 x 8 x 8 cells.  Order 1 in FP32-mixed on
// 4 x 4 x 32 tiles uses a halo of 1 and row pitches of 40 words: 81.6 KB a
// tile, so two 256-thread CTAs share an SM and one's staging and flush
// overlap the other's particles.
template <int MX, int MY, int MZ, int EP, int JP, int H_ = 2, int THREADS = 512, int MINB = 1> struct Layout {
    static constexpr int H = H_;
    static constexpr int kThreads = THREADS, kMinBlocks = MINB;
    static constexpr int EX = MX + 2 * H, EY = MY + 2 * H, EZ = MZ + 2 * H;
    static constexpr int eY = EP, eX = EY * EP, eVol = EX * EY * EP;
    static constexpr int JX = MX + 2 * H + 1, JY = MY + 2 * H + 1, JZ = MZ + 8;
    static constexpr int jY = JP, jX = JY * JP, jVol = JX * JY * JP;
    static_assert(EP >= EZ && JP >= JZ && JP % 4 == 0 && H >= 1 && H <= 2, "row pitches, halo");
    // FP64: J box of doubles (3 components); FP32-mixed: J box of fixed-point
    // (lo, hi) int32 pairs (3 components x 2 arrays)
    template <typename R> static constexpr size_t smem_bytes() {
        return sizeof(R) == 8 ? 8 * (6 * size_t(eVol) + 3 * size_t(jVol)) : 4 * (6 * size_t(eVol) + 6 * size_t(jVol));
    }
};
// FP64 keeps compact pitches: the bank-conflict-free ones would not fit its
// shared memory, and the FP64 path is bound by FP64 arithmetic.
template <typename R>
using LayoutRow = std::conditional_t<sizeof(R) == 4, Layout<4, 4, 32, 64, 64, 2, 512, 1>,
                                     Layout<4, 4, 32, 38, 40, 2, 256, 1>>;
// 8x8x8 tiles: the 32 cells of a warp are 4 z-rows of 8; FP32-mixed row
// pitches of 24 words put those rows on banks 0, 24, 16 and 8 (mod 32), so
// rows never share a bank at the same z.  FP64 keeps compact pitches.
template <typename R>
using LayoutCube = std::conditional_t<sizeof(R) == 4, Layout<8, 8, 8, 24, 24, 2, 512, 1>,
                                      Layout<8, 8, 8, 14, 20, 2, 256, 1>>;
// Order 1, FP32-mixed, 4 x 4 x 32 tiles: halo 1, two CTAs of 256 threads per SM.
using LayoutRow1 = Layout<4, 4, 32, 40, 40, 1, 256, 2>;

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
// (li + H + b_x, lj + H + b_y, lk + 4 + b_z) in box coordinates.  NARROW: all
// three axes have both shapes starting at node b, so the stencil is P cumulative
// slots by (P + 1)^2 transverse nodes (the skipped slots hold exact zeros and,
// on the cumulative axis, the rounding residue of sum dS = 0).
template <int P, typename R, class LY, bool NARROW>
__device__ __forceinline__ void tile_deposit(const StepArgs<R>& A, R* sJ, int li, int lj, int lk,
                                             const EsirkAxis<P, R> ax[3], R wq) {
    constexpr int NC = NARROW ? P : P + 1;
    constexpr int NT = NARROW ? P + 1 : P + 2;
    const R coef[3] = {A.jc[0] * wq, A.jc[1] * wq, A.jc[2] * wq};
    const int bx = li + LY::H + ax[0].b, by = lj + LY::H + ax[1].b, bz = lk + 4 + ax[2].b;
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

// Periodic index of a cell at most one period outside [0, n) (any i, n > 0,
// without a division in that common case).
__device__ __forceinline__ int wrap_near(int i, int n) {
    if (i < 0) i += n;
    else if (i >= n) i -= n;
    return unsigned(i) < unsigned(n) ? i : wrap_any(i, n);
}

// Stage the sub-box [a0,a1) x [b0,b1) x [k0,k1) of the tile's E/B block (cells
// [-H, T+H) per axis around the tile origin oi, oj, ok), periodic wrap in x, y
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
        const int gi = wrap_near(oi - LY::H + a, g.n[0]);
        const int gj = wrap_near(oj - LY::H + b, g.n[1]);
        const int kz = ok - LY::H + kk;
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
// bytes and covers [ok - 4, ok + T + H)).  The box starts at z = ok - 4 (TMA
// wants the innermost coordinate on a 16-byte boundary), so the block is
// addressed 4 - H values in; coordinates outside the grid read as zero and the
// wrapped halo planes are restaged by stage_box after the copy has landed.
constexpr int kTmaSpinLimit = 1 << 20;

template <class LY, typename R> __host__ __device__ constexpr bool tma_layout() {
    return (LY::eY * sizeof(R)) % 16 == 0 && LY::EZ + 4 - LY::H <= LY::eY && LY::eY <= 256;
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
// float4 reductions into HBM); every group read is cleared, so the box is
// zero again for the next tile.  JYc, Q4c > 0: the box extents are the
// layout's (compile-time divisors); 0: the runtime jy, q4.
template <typename R, class LY, int JYc, int Q4c>
__device__ __forceinline__ void flush_fixed4(const StepArgs<R>& A, int* sJi, int oi, int oj, int ok, int jx,
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
        int4* plo = reinterpret_cast<int4*>(sJi + o);
        int4* phi = reinterpret_cast<int4*>(sJi + o + LY::jVol);
        const int4 lo = *plo;
        const int4 hi = *phi;
        if ((lo.x | lo.y | lo.z | lo.w | hi.x | hi.y | hi.z | hi.w) == 0) continue;
        *plo = make_int4(0, 0, 0, 0);
        *phi = make_int4(0, 0, 0, 0);
        // a group of 4 starts at a multiple of 4 and nz % 4 == 0: it is all inside or all beyond the z ends
        if (g.zopen && unsigned(ok - 4 + 4 * q) >= unsigned(g.n[2])) continue;
        const float4 v = make_float4(fixed_to_float(hi.x, fixed_low(hi.x, lo.x)) * A.inv_vscale,
                                     fixed_to_float(hi.y, fixed_low(hi.y, lo.y)) * A.inv_vscale,
                                     fixed_to_float(hi.z, fixed_low(hi.z, lo.z)) * A.inv_vscale,
                                     fixed_to_float(hi.w, fixed_low(hi.w, lo.w)) * A.inv_vscale);
        const int gi = wrap_near(oi - LY::H + a, g.n[0]);
        const int gj = wrap_near(oj - LY::H + b, g.n[1]);
        const int gk = wrap_near(ok - 4 + 4 * q, g.n[2]);
        PIC_CHECK_OR(gk + 3 < g.n[2] && ((gk & 3) == 0), A.err, 6, gk, continue);
        float* dst = reinterpret_cast<float*>(A.J[c]) + ((int64_t)gi * g.n[1] + gj) * g.n[2] + gk;
        atomicAdd(reinterpret_cast<float4*>(dst), v);
    }
}

// Flush of the tile's J box into the global arrays (periodic fold), clearing
// every value it reads.
template <typename R, class LY>
__device__ __forceinline__ void flush_tile(const StepArgs<R>& A, R* sJ, int oi, int oj, int ok) {
    const Geom& g = A.g;
    constexpr bool kFixed = sizeof(R) == 4;
    int* sJi = reinterpret_cast<int*>(sJ);
    const int jx = g.T[0] + 2 * LY::H + 1, jy = g.T[1] + 2 * LY::H + 1, jz = g.T[2] + 8;
    if (kFixed && (g.T[2] % 4) == 0 && (g.n[2] % 4) == 0) {
        // the layout's own tile shape indexes the J box with constants
        if (jx == LY::JX && jy == LY::JY && jz == LY::JZ)
            flush_fixed4<R, LY, LY::JY, LY::JZ / 4>(A, sJi, oi, oj, ok, jx, jy, jz / 4);
        else
            flush_fixed4<R, LY, 0, 0>(A, sJi, oi, oj, ok, jx, jy, jz / 4);
        return;
    }
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
        if (kFixed) {
            int* plo = sJi + 2 * c * LY::jVol + o;
            int* phi = plo + LY::jVol;
            const int lo = *plo, hi = *phi;
            if ((lo | hi) == 0) continue;
            *plo = 0;
            *phi = 0;
            v = R(fixed_to_float(hi, fixed_low(hi, lo)) * A.inv_vscale);
        } else {
            R* pv = sJ + c * LY::jVol + o;
            v = *pv;
            if (v == R(0)) continue;
            *pv = R(0);
        }
        if (g.zopen && unsigned(ok - 4 + kk) >= unsigned(g.n[2])) continue;
        const int gi = wrap_near(oi - LY::H + a, g.n[0]);
        const int gj = wrap_near(oj - LY::H + b, g.n[1]);
        const int gk = wrap_near(ok - 4 + kk, g.n[2]);
        atomicAdd(A.J[c] + ((int64_t)gi * g.n[1] + gj) * g.n[2] + gk, v);
    }
}

// Zero the whole J box (once per CTA: afterwards each flush clears what it reads).
template <typename R, class LY> __device__ __forceinline__ void zero_jbox(R* sJ) {
    const int n16 = sizeof(R) == 4 ? 6 * LY::jVol / 4 : 3 * LY::jVol / 2;
    for (int e = threadIdx.x; e < n16; e += blockDim.x) reinterpret_cast<int4*>(sJ)[e] = make_int4(0, 0, 0, 0);
}

// How one tile's particles are split over the CTA's warps.  The tile's
// particles are cell-sorted; consecutive lanes take consecutive runs of them,
// so the lanes of a warp work in neighbouring cells (distinct shared-memory
// banks).  When the tile's cells split evenly over the warps and the
// particles are spread evenly enough (no warp's share above 1.25x the mean +
// 32), warp w owns the w-th group of cells (z-rows of the 4 x 4 x 32 tile)
// and its lanes split that group's particles: no two warps then deposit into
// the same row at the same time.  Otherwise the whole tile is cut into runs
// of about one cell's worth (or A.run).  Per-warp values.
struct TileWork {
    int beg, end;                              // the tile's particles
    int wbeg, wend, run, nrun, rstart, rstride;
};

template <typename R>
__device__ __forceinline__ void plan_tile(const StepArgs<R>& A, int t, TileWork& w) {
    const Geom& g = A.g;
    w.beg = A.offsets[(int64_t)t * g.cpt];
    w.end = A.offsets[(int64_t)(t + 1) * g.cpt];
    const int cnt = w.end - w.beg;
    const int lane = threadIdx.x & 31;
    const int nwarp = blockDim.x >> 5;
    w.wbeg = w.beg;
    w.wend = w.end;
    bool by_warp = false;
    if (A.run <= 0 && g.cpt % nwarp == 0 && nwarp <= 32) {
        const int cpw = g.cpt / nwarp;
        const int64_t c0 = (int64_t)t * g.cpt;
        const int gsize =
            lane < nwarp ? A.offsets[c0 + (int64_t)(lane + 1) * cpw] - A.offsets[c0 + (int64_t)lane * cpw] : 0;
        const int gmax = __reduce_max_sync(0xffffffffu, gsize);
        by_warp = int64_t(gmax) * nwarp * 4 <= int64_t(cnt) * 5 + int64_t(128) * nwarp;
        if (by_warp) {
            const int wid = threadIdx.x >> 5;
            w.wbeg = A.offsets[c0 + (int64_t)wid * cpw];
            w.wend = A.offsets[c0 + (int64_t)(wid + 1) * cpw];
            PIC_CHECK_OR(w.beg <= w.wbeg && w.wbeg <= w.wend && w.wend <= w.end, A.err, 1,
                         ((long long)w.wbeg << 32) | unsigned(w.wend), w.wbeg = w.wend = w.beg);
        }
    }
    if (by_warp) {
        w.run = max(1, (w.wend - w.wbeg + 31) >> 5);
        w.nrun = (w.wend - w.wbeg + w.run - 1) / w.run;  // at most 32: one pass of the warp
        w.rstart = 0;
        w.rstride = 32;
    } else {
        w.run = A.run > 0 ? A.run : max(1, (cnt + (g.cpt >> 1)) / g.cpt);
        w.nrun = (cnt + w.run - 1) / w.run;
        w.rstart = threadIdx.x - lane;
        w.rstride = blockDim.x;
    }
}

// This lane's first particle of a tile (its loads issued early; see tile_particles).
template <typename R>
__device__ __forceinline__ void first_particle(const StepArgs<R>& A, const TileWork& w, RawParticle<R>& next) {
    const int lane = threadIdx.x & 31;
    const int rr = w.rstart + lane;
    const int p0 = w.wbeg + rr * w.run;
    if (rr < w.nrun && p0 < w.wend) load_raw<R>(A, p0, next);
}

// Gather + push + advance + Esirkepov of one tile's particles, reading E/B from
// the staged block and depositing into the J box.  `next` holds this lane's
// first particle (first_particle).  Warps step their lanes' runs in
// lockstep.  A move whose old and new shapes start on the same node along
// every axis (most moves: crossing a cell face is rare) deposits the narrow
// stencil at once; the others go to a per-warp queue held one slot per lane
// in registers and are deposited 32 at a time with the full window, so
// neither kind runs with idle lanes.
// decode_particle for a particle of tile t (origin oi, oj, ok): in FP32-mixed
// a key inside the tile is unpacked with shifts and masks alone; a key of
// another tile (an outsider, only between sorts) takes the full decode.
template <typename R>
__device__ __forceinline__ void decode_in_tile(const StepArgs<R>& A, const RawParticle<R>& r, int t, int oi, int oj,
                                               int ok, int cell[3], R f0[3], double xg0[3], R u[3], R& wq) {
    if constexpr (sizeof(R) == 4) {
        const Geom& g = A.g;
        const int kk = r.key - g.kbase;
        const int ls = g.lT[1] + g.lT[2];
        if ((kk >> (g.lT[0] + ls)) == t) {
            const int l = kk & (g.cpt - 1);
            cell[0] = oi + (l >> ls);
            cell[1] = oj + ((l >> g.lT[2]) & (g.T[1] - 1));
            cell[2] = ok + (l & (g.T[2] - 1));
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                f0[a] = r.a[a];
                xg0[a] = 0.0;
            }
            u[0] = r.a[3];
            u[1] = r.a[4];
            u[2] = r.a[5];
            wq = r.a[6];
            return;
        }
    }
    decode_particle<R>(A, r, cell, f0, xg0, u, wq);
}

template <int P, typename R, class LY>
__device__ __forceinline__ void tile_particles(const StepArgs<R>& A, const TileWork& w, int t, int oi, int oj, int ok,
                                               const R* sEB, R* sJ, RawParticle<R> next) {
    const Geom& g = A.g;
    constexpr bool kFixed = sizeof(R) == 4;
    const int lane = threadIdx.x & 31;
    TileMove<R> qs = TileMove<R>::zero();  // this lane's queue slot
    int qn = 0;                            // queued moves (warp-uniform)
    for (int rbase = w.rstart; rbase < w.nrun; rbase += w.rstride) {
        const int rr = rbase + lane;
        const int p0 = w.wbeg + rr * w.run;
        const int len = rr < w.nrun ? min(w.run, w.wend - p0) : 0;
        const int maxlen = __reduce_max_sync(0xffffffffu, len);
        // the next particle's loads are issued before the current one's work;
        // `next` holds this run's first particle (loaded by first_particle or
        // during the previous run), and the last particle of a run prefetches
        // the next run's first
        const int rr_n = rr + w.rstride;
        const int p0_n = w.wbeg + rr_n * w.run;
        const bool has_n = rr_n < w.nrun && p0_n < w.wend;
        if (len == 0 && has_n) load_raw<R>(A, p0_n, next);
        for (int it = 0; it < maxlen; ++it) {
            const int p = p0 + it;
            bool wide = false;
            TileMove<R> mine = TileMove<R>::zero();
            const RawParticle<R> raw = next;
            if (it + 1 < len) load_raw<R>(A, p + 1, next);
            else if (it + 1 == len && has_n) load_raw<R>(A, p0_n, next);
            if (it < len) {
                int cell[3];
                R f0[3], u[3], wq;
                double xg0[3];
                decode_in_tile<R>(A, raw, t, oi, oj, ok, cell, f0, xg0, u, wq);
                const int li = cell[0] - oi, lj = cell[1] - oj, lk = cell[2] - ok;
                // the fixed-point sums are exact for up to 65535 particles per tile
                const bool inside = unsigned(li) < unsigned(g.T[0]) && unsigned(lj) < unsigned(g.T[1]) &&
                                    unsigned(lk) < unsigned(g.T[2]) && (!kFixed || p - w.beg < 65535);
                if (!inside) {
                    const int slot = atomicAdd(A.outn, 1);
                    A.outl[slot] = p;
                } else {
                    if (A.perm) {
                        // a sorted-order step writes the whole particle into its
                        // slot: id and weight here, the rest in store_particle
                        A.did[p] = raw.id;
                        A.pa[6][p] = raw.a[6];
                    }
                    R EB[6];
                    {
                        GatherW<P, R> G;
                        int fn[3], fs[3];
                        gather_weights<P, R>(f0, G, fn, fs, A.egather != 0);
                        constexpr int H = LY::H;
                        const int bnx = (li + H + fn[0]) * LY::eX, bsx = (li + H + fs[0]) * LY::eX;
                        const int bny = (lj + H + fn[1]) * LY::eY, bsy = (lj + H + fs[1]) * LY::eY;
                        const int bnz = lk + H + fn[2], bsz = lk + H + fs[2];
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
                        keep_particle<R>(A, p, raw);
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
}

// Whether tile t stages its E/B block by TMA: the layout allows it, a
// descriptor exists, the block is 128-byte aligned and the box's z start
// (ok - 4) is on a 16-byte boundary.
template <typename R, class LY>
__device__ __forceinline__ bool tile_uses_tma(const CUtensorMap* tmap, const R* sm, int ok) {
    if constexpr (!tma_layout<LY, R>()) return false;
    return tmap != nullptr && (unsigned(__cvta_generic_to_shared(sm)) & 127u) == 0u && ((ok - 4) & 3) == 0;
}

// Halo planes of a TMA-staged block that wrap around the grid came in as
// zeros: restage them by loads.
template <typename R, class LY>
__device__ __forceinline__ void restage_wrapped(const StepArgs<R>& A, R* sEB, int oi, int oj, int ok) {
    const Geom& g = A.g;
    constexpr int H = LY::H;
    const int ex = g.T[0] + 2 * H, ey = g.T[1] + 2 * H, ez = g.T[2] + 2 * H;
    if (oi < H) stage_box<R, LY>(A, sEB, oi, oj, ok, 0, H - oi, 0, ey, 0, ez);
    if (oi + ex - H > g.n[0]) stage_box<R, LY>(A, sEB, oi, oj, ok, g.n[0] - oi + H, ex, 0, ey, 0, ez);
    if (oj < H) stage_box<R, LY>(A, sEB, oi, oj, ok, 0, ex, 0, H - oj, 0, ez);
    if (oj + ey - H > g.n[1]) stage_box<R, LY>(A, sEB, oi, oj, ok, 0, ex, g.n[1] - oj + H, ey, 0, ez);
    if (!g.zopen) {
        if (ok < H) stage_box<R, LY>(A, sEB, oi, oj, ok, 0, ex, 0, ey, 0, H - ok);
        if (ok + ez - H > g.n[2]) stage_box<R, LY>(A, sEB, oi, oj, ok, 0, ex, 0, ey, g.n[2] - ok + H, ez);
    }
}

// Stage the whole block by loads.
template <typename R, class LY>
__device__ __forceinline__ void stage_all(const StepArgs<R>& A, R* sEB, int oi, int oj, int ok) {
    const Geom& g = A.g;
    const int ex = g.T[0] + 2 * LY::H, ey = g.T[1] + 2 * LY::H, ez = g.T[2] + 2 * LY::H;
    if (ex == LY::EX && ey == LY::EY && ez == LY::EZ)
        stage_box<R, LY, true>(A, sEB, oi, oj, ok, 0, ex, 0, ey, 0, ez);
    else
        stage_box<R, LY>(A, sEB, oi, oj, ok, 0, ex, 0, ey, 0, ez);
}

// Next tile with particles from the queue (one thread), or -1 when none is left.
__device__ __forceinline__ int next_tile(const int* __restrict__ offsets, int cpt, int ntiles, int* queue) {
    for (;;) {
        const int t = atomicAdd(queue, 1);
        if (t >= ntiles) return -1;
        if (offsets[(int64_t)(t + 1) * cpt] > offsets[(int64_t)t * cpt]) return t;
    }
}

// Persistent tile loop of one box: each CTA pulls tiles from a queue counter
// (zeroed before the launch) and pipelines them.  While it flushes tile t's
// current, the TMA copy of tile t+1's E/B block is already in flight (the
// gather of t is done with the block) and each lane's first particle of t+1
// is loading; the flush clears the J box as it reads it, so no zeroing pass is
// needed between tiles.  The E/B block is free once every warp has finished
// tile t's particles; the J box once the flush is done.
template <int P, typename R, class LY>
__device__ __forceinline__ void tile_loop(const StepArgs<R>& A, int* queue, unsigned char* smem_raw,
                                          const CUtensorMap* tmap) {
    R* sm = reinterpret_cast<R*>(smem_raw);
    const Geom& g = A.g;
    constexpr int kZShift = tma_layout<LY, R>() ? 4 - LY::H : 0;
    R* sEB = sm + kZShift;
    R* sJ = sm + 6 * LY::eVol;
    const int ntiles = int(g.ntiles);
    __shared__ __align__(8) unsigned long long s_bar;
    __shared__ int s_tile[2];

    zero_jbox<R, LY>(sJ);
    if (threadIdx.x == 0) {
        mbar_init(&s_bar);
        s_tile[0] = next_tile(A.offsets, g.cpt, ntiles, queue);
    }
    __syncthreads();
    int t = s_tile[0];
    if (t < 0) {
        if (threadIdx.x == 0) mbar_inval(&s_bar);
        return;
    }
    int oi, oj, ok;
    tile_origin(g, t, oi, oj, ok);
    TileWork w;
    plan_tile<R>(A, t, w);
    RawParticle<R> next;
    first_particle<R>(A, w, next);
    bool by_tma = tile_uses_tma<R, LY>(tmap, sm, ok);
    if (by_tma) {
        if (threadIdx.x == 0)
            tma_load_eb(tmap, sm, &s_bar, unsigned(6 * LY::eVol * sizeof(R)), ok - 4, oj - LY::H, oi - LY::H);
    } else {
        stage_all<R, LY>(A, sEB, oi, oj, ok);
    }
    unsigned phase = 0;  // parity of the barrier phase the next TMA copy completes
    for (;;) {
        if (threadIdx.x == 0) s_tile[1] = next_tile(A.offsets, g.cpt, ntiles, queue);
        if (by_tma) {
            // every thread waits for the copy; if it did not land in time, all
            // wait once more (it is still writing into this CTA's shared
            // memory), then the CTA stops: its block cannot be reused safely
            const bool late = __syncthreads_or(!mbar_wait(&s_bar, phase, kTmaSpinLimit));
            if (late) {
                if (threadIdx.x == 0) raise_error(A.err, ERRBIT_TIMEOUT);
                mbar_wait(&s_bar, phase, kTmaSpinLimit);
                __syncthreads();
                return;
            }
            phase ^= 1u;
            restage_wrapped<R, LY>(A, sEB, oi, oj, ok);
        }
        __syncthreads();  // E/B of t staged; s_tile[1] visible
        PIC_CHECK_OR(w.beg >= 0 && w.end <= A.np, A.err, 1, ((long long)w.beg << 32) | unsigned(w.end),
                     w.wbeg = w.wend = w.beg);
        tile_particles<P, R, LY>(A, w, t, oi, oj, ok, sEB, sJ, next);
        __syncthreads();  // every warp is done with t's E/B block and deposits
        const int tn = s_tile[1];
        int ni = 0, nj = 0, nk = 0;
        bool tma_n = false;
        if (tn >= 0) {
            tile_origin(g, tn, ni, nj, nk);
            tma_n = tile_uses_tma<R, LY>(tmap, sm, nk);
            if (tma_n && threadIdx.x == 0)
                tma_load_eb(tmap, sm, &s_bar, unsigned(6 * LY::eVol * sizeof(R)), nk - 4, nj - LY::H, ni - LY::H);
            plan_tile<R>(A, tn, w);
            first_particle<R>(A, w, next);
        }
        flush_tile<R, LY>(A, sJ, oi, oj, ok);
        if (tn >= 0 && !tma_n) stage_all<R, LY>(A, sEB, ni, nj, nk);
        if (tn < 0) break;
        __syncthreads();  // J box clear; a load-staged block complete
        t = tn;
        oi = ni, oj = nj, ok = nk;
        by_tma = tma_n;
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_inval(&s_bar);
}

template <int P, typename R, class LY>
__global__ void __launch_bounds__(LY::kThreads, LY::kMinBlocks)
    k_tile_step(StepArgs<R> A, const __grid_constant__ CUtensorMap tmap, int use_tma, int* queue) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    tile_loop<P, R, LY>(A, queue, smem_raw, use_tma ? &tmap : nullptr);
}

// Next (box, tile) work item with particles from the queue (one thread), or
// -1 when none is left.
template <typename R>
__device__ __forceinline__ int next_item(const StepArgs<R>* __restrict__ boxes, const int2* __restrict__ items,
                                         int nitems, int* queue) {
    for (;;) {
        const int it = atomicAdd(queue, 1);
        if (it >= nitems) return -1;
        const int2 bt = items[it];
        const StepArgs<R>& B = boxes[bt.x];
        const int cpt = B.g.cpt;
        if (B.offsets[(int64_t)(bt.y + 1) * cpt] > B.offsets[(int64_t)bt.y * cpt]) return it;
    }
}

// A box's arguments into a shared-memory slot (all threads).
template <typename R> __device__ __forceinline__ void copy_args(const StepArgs<R>* src, StepArgs<R>* dst) {
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    for (int w = threadIdx.x; w < int(sizeof(StepArgs<R>) / 4); w += blockDim.x) d[w] = s[w];
}

// Batch of boxes: a persistent grid pulls (box, tile) items, heaviest first,
// from a queue counter (zeroed before the launch) and pipelines them as
// tile_loop does; the box arguments of the current and the next item sit in
// two shared-memory slots, the next item's copied while the current one's
// current is flushed.
template <int P, typename R, class LY>
__global__ void __launch_bounds__(LY::kThreads, LY::kMinBlocks)
    k_tile_step_batch(const StepArgs<R>* __restrict__ boxes, const int2* __restrict__ items, int nitems, int* queue) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(16) StepArgs<R> sA[2];
    __shared__ __align__(8) unsigned long long s_bar;
    __shared__ int s_item[2];
    R* sm = reinterpret_cast<R*>(smem_raw);
    constexpr int kZShift = tma_layout<LY, R>() ? 4 - LY::H : 0;
    R* sEB = sm + kZShift;
    R* sJ = sm + 6 * LY::eVol;

    zero_jbox<R, LY>(sJ);
    if (threadIdx.x == 0) {
        mbar_init(&s_bar);
        s_item[0] = next_item<R>(boxes, items, nitems, queue);
    }
    __syncthreads();
    int it = s_item[0];
    if (it < 0) {
        if (threadIdx.x == 0) mbar_inval(&s_bar);
        return;
    }
    int slot = 0;
    copy_args<R>(boxes + items[it].x, &sA[0]);
    __syncthreads();
    int t = items[it].y;
    int oi, oj, ok;
    tile_origin(sA[0].g, t, oi, oj, ok);
    TileWork w;
    plan_tile<R>(sA[0], t, w);
    RawParticle<R> next;
    first_particle<R>(sA[0], w, next);
    bool by_tma = tile_uses_tma<R, LY>(sA[0].tmap, sm, ok);
    if (by_tma) {
        if (threadIdx.x == 0)
            tma_load_eb(sA[0].tmap, sm, &s_bar, unsigned(6 * LY::eVol * sizeof(R)), ok - 4, oj - LY::H, oi - LY::H);
    } else {
        stage_all<R, LY>(sA[0], sEB, oi, oj, ok);
    }
    unsigned phase = 0;
    for (;;) {
        const StepArgs<R>& A = sA[slot];
        if (threadIdx.x == 0) s_item[1] = next_item<R>(boxes, items, nitems, queue);
        if (by_tma) {
            const bool late = __syncthreads_or(!mbar_wait(&s_bar, phase, kTmaSpinLimit));
            if (late) {  // as in tile_loop: the CTA stops
                if (threadIdx.x == 0) raise_error(A.err, ERRBIT_TIMEOUT);
                mbar_wait(&s_bar, phase, kTmaSpinLimit);
                __syncthreads();
                return;
            }
            phase ^= 1u;
            restage_wrapped<R, LY>(A, sEB, oi, oj, ok);
        }
        __syncthreads();  // E/B of t staged; s_item[1] visible
        tile_particles<P, R, LY>(A, w, t, oi, oj, ok, sEB, sJ, next);
        __syncthreads();  // every warp is done with t's block and deposits
        const int itn = s_item[1];
        int tn = -1, ni = 0, nj = 0, nk = 0;
        bool tma_n = false;
        if (itn >= 0) {
            const int2 bt = items[itn];
            const StepArgs<R>& An = boxes[bt.x];  // read from global until its slot is filled
            tn = bt.y;
            tile_origin(An.g, tn, ni, nj, nk);
            tma_n = tile_uses_tma<R, LY>(An.tmap, sm, nk);
            if (tma_n && threadIdx.x == 0)
                tma_load_eb(An.tmap, sm, &s_bar, unsigned(6 * LY::eVol * sizeof(R)), nk - 4, nj - LY::H, ni - LY::H);
            plan_tile<R>(An, tn, w);
            first_particle<R>(An, w, next);
            copy_args<R>(boxes + bt.x, &sA[1 - slot]);
        }
        flush_tile<R, LY>(A, sJ, oi, oj, ok);
        if (itn >= 0 && !tma_n) stage_all<R, LY>(boxes[items[itn].x], sEB, ni, nj, nk);
        if (itn < 0) break;
        __syncthreads();  // J box clear, next slot filled, a load-staged block complete
        slot = 1 - slot;
        t = tn;
        oi = ni, oj = nj, ok = nk;
        by_tma = tma_n;
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_inval(&s_bar);
}

// One particle the tile kernel listed as outside its tile: gather from global
// memory, push, deposit with global atomics (the same arithmetic).
template <int P, typename R>
__device__ __forceinline__ void outsider_body(const StepArgs<R>& A, const int p) {
    int cell[3];
    R f0[3], u[3], wq;
    double xg0[3];
    RawParticle<R> raw;
    load_raw<R>(A, p, raw);
    decode_particle<R>(A, raw, cell, f0, xg0, u, wq);
    if (A.perm) {  // id and weight into the slot (store_particle writes the rest)
        A.did[p] = raw.id;
        A.pa[6][p] = raw.a[6];
    }
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
        keep_particle<R>(A, p, raw);
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

// Persistent CTAs of the tile kernel: as many as fit on the GPU at once (the
// SM count times the CTAs per SM the kernel's resources allow), at most one
// per tile.
template <typename R, int P, class LY> int tile_grid(const pic_ctx* c) {
    static int per_sm = 0;  // per instantiation; found outside stream capture by pic_init_grid
    if (per_sm == 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tile_step<P, R, LY>, LY::kThreads,
                                                          LY::template smem_bytes<R>()) != cudaSuccess ||
            n < 1) {
            cudaGetLastError();
            n = 1;
        }
        per_sm = n;
    }
    const int64_t g = int64_t(c->sms) * per_sm;
    return int(g < c->g.ntiles ? g : c->g.ntiles);
}

template <typename R, int P, class LY> cudaError_t tile_step_impl(pic_ctx* c) {
    // after a permutation sort the kernel moves the particles from the other
    // buffer into the current one in sorted order (the step's sort handed over)
    StepArgs<R> A = c->tile_perm ? make_args_perm<R>(c, 1 - c->cur, c->cur, c->perm) : make_args<R>(c);
    const size_t smem = LY::template smem_bytes<R>();
    // the tile queue counter sits after the outsider count (zeroed with it)
    int* queue = reinterpret_cast<int*>(c->err + 5);
    const bool filt = c->filter_passes > 0 && c->Fg;
    k_tile_step<P, R, LY><<<unsigned(tile_grid<R, P, LY>(c)), LY::kThreads, smem, c->stream>>>(
        A, filt ? c->tmap_g : c->tmap_eb, (filt ? c->tma_g : c->tma) ? 1 : 0, queue);
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
    if constexpr (sizeof(R) == 4)
        if (c->layout == 2) return tile_step_impl<float, 1, LayoutRow1>(c);
    return c->layout == 1 ? tile_step_order<R, LayoutRow<R>>(c) : tile_step_order<R, LayoutCube<R>>(c);
}

cudaError_t launch_tile_step(pic_ctx* c) {
    // J is one allocation of three components (see pic_api.cu); the outsider
    // count and the tile queue counter sit after the four error words
    cudaError_t e = cudaMemsetAsync(c->j_other ? c->Fo[6] : c->F[6], 0, 3 * c->g.C * c->rsize, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err + 4, 0, 2 * sizeof(unsigned), c->stream);
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
    if (layout == 2 && f64) return false;  // the halo-1 layout is FP32-mixed only
    const cuuint32_t bz = layout == 2 ? LayoutRow1::eY
                          : layout == 1 ? (f64 ? LayoutRow<double>::eY : LayoutRow<float>::eY)
                                        : (f64 ? LayoutCube<double>::eY : LayoutCube<float>::eY);
    // x, y extents are the same for both precisions
    const cuuint32_t by = layout == 2 ? LayoutRow1::EY : layout == 1 ? LayoutRow<float>::EY : LayoutCube<float>::EY;
    const cuuint32_t bx = layout == 2 ? LayoutRow1::EX : layout == 1 ? LayoutRow<float>::EX : LayoutCube<float>::EX;
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
    c->tma = encode_eb_tensor_map(&c->tmap_eb, c->F[0], c->g.n, c->g.C, c->layout, c->prec);
    c->tma_o = c->Fo[0] && encode_eb_tensor_map(&c->tmap_eb_o, c->Fo[0], c->g.n, c->g.C, c->layout, c->prec);
}

void swap_field_sets(pic_ctx* c) {
    for (int i = 0; i < 9; ++i) std::swap(c->F[i], c->Fo[i]);
    std::swap(c->tmap_eb, c->tmap_eb_o);
    std::swap(c->tma, c->tma_o);
    c->fpar ^= 1;
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
    PIC_CFG(float, 1, LayoutRow1)
    PIC_CFG(float, 1, LayoutRow<float>) PIC_CFG(float, 2, LayoutRow<float>) PIC_CFG(float, 3, LayoutRow<float>)
    PIC_CFG(float, 1, LayoutCube<float>) PIC_CFG(float, 2, LayoutCube<float>) PIC_CFG(float, 3, LayoutCube<float>)
    PIC_CFG(double, 1, LayoutRow<double>) PIC_CFG(double, 2, LayoutRow<double>) PIC_CFG(double, 3, LayoutRow<double>)
    PIC_CFG(double, 1, LayoutCube<double>) PIC_CFG(double, 2, LayoutCube<double>) PIC_CFG(double, 3, LayoutCube<double>)
#undef PIC_CFG
    // the persistent grids' CTAs per SM, found now (outside any stream capture)
    if (e == cudaSuccess) {
        switch (c->order) {
        case 1:
            if (c->prec == PIC_FP64) (void)(c->layout == 1 ? tile_grid<double, 1, LayoutRow<double>>(c)
                                                           : tile_grid<double, 1, LayoutCube<double>>(c));
            else (void)(c->layout == 2   ? tile_grid<float, 1, LayoutRow1>(c)
                        : c->layout == 1 ? tile_grid<float, 1, LayoutRow<float>>(c)
                                         : tile_grid<float, 1, LayoutCube<float>>(c));
            break;
        case 2:
            if (c->prec == PIC_FP64) (void)(c->layout == 1 ? tile_grid<double, 2, LayoutRow<double>>(c)
                                                           : tile_grid<double, 2, LayoutCube<double>>(c));
            else (void)(c->layout == 1 ? tile_grid<float, 2, LayoutRow<float>>(c)
                                       : tile_grid<float, 2, LayoutCube<float>>(c));
            break;
        default:
            if (c->prec == PIC_FP64) (void)(c->layout == 1 ? tile_grid<double, 3, LayoutRow<double>>(c)
                                                           : tile_grid<double, 3, LayoutCube<double>>(c));
            else (void)(c->layout == 1 ? tile_grid<float, 3, LayoutRow<float>>(c)
                                       : tile_grid<float, 3, LayoutCube<float>>(c));
        }
    }
    return e;
}

// ---- batch of boxes ----------------------------------------------------------
template <typename R, int P> cudaError_t tile_batch_impl(const BatchTileLaunch& L, cudaStream_t s) {
    using LY = LayoutCube<R>;
    if (L.nitems <= 0) return cudaSuccess;
    const size_t smem = LY::template smem_bytes<R>();
    const int grid = L.grid < L.nitems ? L.grid : L.nitems;
    k_tile_step_batch<P, R, LY><<<unsigned(grid), LY::kThreads, smem, s>>>(
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
