// Support kernels of libpic around the fused tile kernel: the Yee update
// (one box and batches of boxes), particle load / store and field
// conversion, diagnostics, the moving window's shift and injection, and the
// re-keying of particles after a change of tile shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "pic_ctx.h"
#include "pic_device.cuh"
#include "pic_step_common.cuh"

namespace pic {

static inline unsigned blocks_for(int64_t n) { return unsigned((n + kBlock - 1) / kBlock); }

// ---------------------------------------------------------------------------
// Yee FDTD
// ---------------------------------------------------------------------------

// B <- B - h curl E (forward differences: B sits half a cell above E), at
// cell (i, j, k) = c.
template <typename R>
__device__ __forceinline__ void yee_b_ijk(const YeeArgs<R>& Y, const int64_t c, const int i, const int j, const int k) {
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

// The cell's indices from its linear index (the batch kernels' one-dimensional blocks).
template <typename R> __device__ __forceinline__ void cell_ijk(const YeeArgs<R>& Y, int64_t c, int& i, int& j, int& k) {
    k = int(c % Y.n[2]);
    j = int((c / Y.n[2]) % Y.n[1]);
    i = int(c / ((int64_t)Y.n[1] * Y.n[2]));
}

template <typename R> __device__ __forceinline__ void yee_b_at(const YeeArgs<R>& Y, const int64_t c) {
    int i, j, k;
    cell_ijk(Y, c, i, j, k);
    yee_b_ijk(Y, c, i, j, k);
}

// CKC (Cole-Karkkainen, the solver named for the plasma-acceleration run,
// Sec. 4.2; cubic cells): the forward difference of F along `axis`, averaged
// over the two transverse axes with weights (1/4, 1/2, 1/4) per axis.  off[a][m]
// is the element offset of coordinate (cell + m - 1) along axis a, wrapped
// periodically; ok[m] is false where that z coordinate lies beyond an open z end
// (the field there is zero).
template <typename R>
__device__ __forceinline__ R ckc_diff(const R* __restrict__ F, int axis, const int64_t off[3][4], const bool ok[4],
                                      R inv) {
    const int t1 = axis == 0 ? 1 : (axis == 1 ? 2 : 0), t2 = axis == 0 ? 2 : (axis == 1 ? 0 : 1);
    const R w[3] = {R(0.25), R(0.5), R(0.25)};
    R acc = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            int m0[3], m1[3];
            m0[axis] = 1, m1[axis] = 2;  // the cell and the next one along the difference
            m0[t1] = m1[t1] = a;
            m0[t2] = m1[t2] = b;
            const R v1 = ok[m1[2]] ? F[off[0][m1[0]] + off[1][m1[1]] + off[2][m1[2]]] : R(0);
            const R v0 = ok[m0[2]] ? F[off[0][m0[0]] + off[1][m0[1]] + off[2][m0[2]]] : R(0);
            acc += w[a] * w[b] * (v1 - v0);
        }
    return acc * inv;
}

template <typename R>
__device__ __forceinline__ void yee_b_ckc_ijk(const YeeArgs<R>& Y, const int64_t c, const int i, const int j,
                                              const int k) {
    const int cc[3] = {i, j, k};
    const int64_t st[3] = {(int64_t)Y.n[1] * Y.n[2], Y.n[2], 1};
    int64_t off[3][4];
    bool ok[4];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            int q = cc[a] + m - 1;  // within one period: n >= 3
            q = q < 0 ? q + Y.n[a] : (q >= Y.n[a] ? q - Y.n[a] : q);
            if (q >= Y.n[a]) q -= Y.n[a];
            off[a][m] = q * st[a];
        }
#pragma unroll
    for (int m = 0; m < 4; ++m) ok[m] = !Y.zopen || unsigned(k + m - 1) < unsigned(Y.n[2]);
    const R dEz_dy = ckc_diff(Y.E[2], 1, off, ok, Y.inv[1]), dEy_dz = ckc_diff(Y.E[1], 2, off, ok, Y.inv[2]);
    const R dEx_dz = ckc_diff(Y.E[0], 2, off, ok, Y.inv[2]), dEz_dx = ckc_diff(Y.E[2], 0, off, ok, Y.inv[0]);
    const R dEy_dx = ckc_diff(Y.E[1], 0, off, ok, Y.inv[0]), dEx_dy = ckc_diff(Y.E[0], 1, off, ok, Y.inv[1]);
    Y.B[0][c] -= Y.h * (dEz_dy - dEy_dz);
    Y.B[1][c] -= Y.h * (dEx_dz - dEz_dx);
    Y.B[2][c] -= Y.h * (dEy_dx - dEx_dy);
}

// E <- E + dt (curl B - J) (backward differences), at cell (i, j, k) = c.
template <typename R>
__device__ __forceinline__ void yee_e_ijk(const YeeArgs<R>& Y, const int64_t c, const int i, const int j, const int k) {
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

template <typename R> __device__ __forceinline__ void yee_e_at(const YeeArgs<R>& Y, const int64_t c) {
    int i, j, k;
    cell_ijk(Y, c, i, j, k);
    yee_e_ijk(Y, c, i, j, k);
}

// Single-box grids: block x is a z-row (i, j) of the grid, block y a chunk of
// kBlock cells along it, so no thread divides a 64-bit cell index.
struct RowCell {
    int i, j, k;
    int64_t c;
    bool ok;
};
template <typename R> __device__ __forceinline__ RowCell row_cell(const YeeArgs<R>& Y) {
    RowCell r;
    const int row = int(blockIdx.x);
    r.i = row / Y.n[1];
    r.j = row - r.i * Y.n[1];
    r.k = int(blockIdx.y) * blockDim.x + threadIdx.x;
    r.ok = r.k < Y.n[2];
    r.c = (int64_t)row * Y.n[2] + r.k;
    return r;
}

template <typename R> __global__ void __launch_bounds__(kBlock) k_yee_b(YeeArgs<R> Y) {
    const RowCell r = row_cell(Y);
    if (Y.step && r.c == 0) *Y.step += 1;
    if (r.ok) yee_b_ijk(Y, r.c, r.i, r.j, r.k);
}

// The B half step with the CKC stencil (a kernel of its own: its register
// needs must not lower the occupancy of the plain Yee update).
template <typename R> __global__ void __launch_bounds__(kBlock, 3) k_yee_b_ckc(YeeArgs<R> Y) {
    const RowCell r = row_cell(Y);
    if (Y.step && r.c == 0) *Y.step += 1;
    if (r.ok) yee_b_ckc_ijk(Y, r.c, r.i, r.j, r.k);
}

template <typename R> __global__ void __launch_bounds__(kBlock) k_yee_e(YeeArgs<R> Y) {
    const RowCell r = row_cell(Y);
    if (r.ok) yee_e_ijk(Y, r.c, r.i, r.j, r.k);
}

// ---------------------------------------------------------------------------
// The whole Yee step in one pass (plain Yee solver), from one field set into
// the other, with the formulas of yee_b_ijk / yee_e_ijk: B half step, E step,
// B half step.  Each block owns a y-z tile of kYTY x kYTZ cells and marches
// along an x-chunk of kYXC cells; at x = i it
//   - computes B'(i+1) = B(i+1) - dt/2 curl E on the tile plus a one-cell
//     y-z halo (needs E at i+1 and i+2),
//   - computes E'(i+1) = E(i+1) + dt (curl B' - J) on the tile plus the
//     halo cell above in y and z (needs B' at i+1 and i),
//   - computes B''(i) = B'(i) - dt/2 curl E' on the tile (needs E' at i and
//     i+1) and writes E'(i) and B''(i) into the other field set.
// Shared memory holds y-z planes only (E: ring of 4, B: ring of 3, J: ring of
// 2), the next planes load with cp.async while the current ones compute, so
// HBM sees E, B, J read once and E, B written once a cell (60 bytes in FP32
// against the three in-place passes' 120); the y-z halos are re-read from L2
// by the neighbouring tiles.  Reads and writes go to different arrays, so no
// block sees another's new values.  With z open, fields beyond the z ends are
// zero in every phase.
//
// Planes are stored row by row (y), 32 cells a row for E (z from k0 - 1), 31
// for B, 30 for J (z from k0): warp w works row w, its lanes along z.
// ---------------------------------------------------------------------------
constexpr int kYTY = 7;                        // tile rows (y)
constexpr int kYTZ = 29;                       // tile depth (z): E rows are 32 cells
constexpr int kEY = kYTY + 3, kEZ = kYTZ + 3;  // E plane: y from -1, z from -1
constexpr int kBY = kYTY + 2, kBZ = kYTZ + 2;  // B plane: y from -1, z from -1
constexpr int kJY = kYTY + 1, kJZ = kYTZ + 1;  // J plane: y from 0, z from 0
constexpr int kEP = kEY * kEZ, kBP = kBY * kBZ, kJP = kJY * kJZ;
constexpr int kYWarps = kEY;                   // warp w stages row w of every plane
constexpr int kYThreads = 32 * kYWarps;
static_assert(kEZ == 32, "E rows are one warp wide");

template <typename R> constexpr size_t yee_fused_smem() { return sizeof(R) * 3 * size_t(4 * kEP + 3 * kBP + 2 * kJP); }

template <typename R> struct YeeFusedArgs {
    const R* E[3];
    const R* B[3];
    const R* J[3];
    R* Eo[3];  // the other set, written
    R* Bo[3];
    int n[3];
    int nt[3];  // x-chunks, y tiles, z tiles
    int xc;     // x-chunk length
    R inv[3];
    R h;   // dt / 2
    R dt;
    long long* step;
    int zopen;
};

// One element copied global -> shared without passing through registers
// (cp.async: every copy of a plane is in flight at once); a source size of 0
// fills the element with zero, the source address stays a valid one.
template <typename R> __device__ __forceinline__ void copy_elem_async(R* dst, const R* src, bool ok) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    const unsigned bytes = ok ? unsigned(sizeof(R)) : 0u;
    if constexpr (sizeof(R) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ int step_wrap(int x, int n) { return x + 1 == n ? 0 : x + 1; }

template <typename R> __global__ void __launch_bounds__(kYThreads) k_yee_fused(YeeFusedArgs<R> Y) {
    extern __shared__ __align__(16) unsigned char yee_raw[];
    R* const sm = reinterpret_cast<R*>(yee_raw);
    R* const Eb = sm;                  // 4 planes x 3 components x kEP
    R* const Bb = Eb + 12 * kEP;       // 3 planes x 3 x kBP
    R* const Jb = Bb + 9 * kBP;        // 2 planes x 3 x kJP
    // z fastest, then y, then the x-chunk: neighbouring tiles run together
    const int bz = int(blockIdx.x % unsigned(Y.nt[2]));
    const int rb = int(blockIdx.x / unsigned(Y.nt[2]));
    const int by = rb % Y.nt[1], bx = rb / Y.nt[1];
    const int x0 = bx * Y.xc, x1 = min(x0 + Y.xc, Y.n[0]);
    const int j0 = by * kYTY, k0 = bz * kYTZ;
    const int warp = int(threadIdx.x) >> 5, lane = int(threadIdx.x) & 31;
    const int64_t sx = int64_t(Y.n[1]) * Y.n[2];
    // this lane's z in the E / B planes (from k0 - 1) and in the J plane (from k0)
    const int zlo = k0 - 1 + lane, zj = k0 + lane;
    const bool zlo_in = unsigned(zlo) < unsigned(Y.n[2]), zj_in = unsigned(zj) < unsigned(Y.n[2]);
    const bool zlo_ok = !Y.zopen || zlo_in, zj_ok = !Y.zopen || zj_in;
    // this thread's row w of the E and B planes (y = j0 - 1 + w) and of the J
    // plane (y = j0 + w): source offsets within an x-plane, wrapped
    const int64_t off_eb = int64_t(wrap_any(j0 - 1 + warp, Y.n[1])) * Y.n[2] + wrap_any(zlo, Y.n[2]);
    const int64_t off_j = int64_t(wrap_any(j0 + warp, Y.n[1])) * Y.n[2] + wrap_any(zj, Y.n[2]);
    const bool ld_b = warp < kBY && lane < kBZ, ld_j = warp < kJY && lane < kJZ;
    const int se = warp * kEZ + lane, sb = warp * kBZ + lane, sj = warp * kJZ + lane;

    // E(xe) into plane eb, B(xb) into bb, J(xj) into jb (x wrapped; a null
    // plane skips that field), row `warp` of every component
    auto load_planes = [&](int xe, R* eb, int xb, R* bb, int xj, R* jb) {
        if (eb) {
            const int64_t o = xe * sx + off_eb;
#pragma unroll
            for (int c = 0; c < 3; ++c) copy_elem_async(eb + c * kEP + se, Y.E[c] + o, zlo_ok);
        }
        if (bb && ld_b) {
            const int64_t o = xb * sx + off_eb;
#pragma unroll
            for (int c = 0; c < 3; ++c) copy_elem_async(bb + c * kBP + sb, Y.B[c] + o, zlo_ok);
        }
        if (jb && ld_j) {
            const int64_t o = xj * sx + off_j;
#pragma unroll
            for (int c = 0; c < 3; ++c) copy_elem_async(jb + c * kJP + sj, Y.J[c] + o, zj_ok);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    // ring roles: E'(i) / E(i+1) -> E'(i+1) / E(i+2) / E(i+3) loading;
    // B'(i) / B(i+1) -> B'(i+1) / B(i+2) loading; J(i+1) / J(i+2) loading
    int eP = 0, eC = 1, eN = 2, eL = 3, b0 = 0, b1 = 1, bL = 2, j1 = 0, jL = 1;
    // the march starts at i = x0 - 2 with E(x0 - 1), E(x0) and B(x0 - 1) in
    int xm = wrap_any(x0 - 1, Y.n[0]);  // x0 - 1, wrapped
    int xz = step_wrap(xm, Y.n[0]);     // x0
    load_planes(xm, Eb + 3 * eC * kEP, xm, Bb + 3 * b1 * kBP, 0, nullptr);
    load_planes(xz, Eb + 3 * eN * kEP, 0, nullptr, 0, nullptr);
    int xb = xz;                        // i + 2 at i = x0 - 2, wrapped
    int xe = step_wrap(xb, Y.n[0]);     // i + 3
    const R h = Y.h;
    for (int i = x0 - 2; i < x1; ++i) {
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();  // this step's planes are in; last step's readers are done
        if (i + 1 < x1)   // E(i+3), B(i+2), J(i+2) for the next step
            load_planes(xe, Eb + 3 * eL * kEP, xb, Bb + 3 * bL * kBP, xb, Jb + 3 * jL * kJP);
        xb = xe;
        xe = step_wrap(xe, Y.n[0]);
        const R* Ec = Eb + 3 * eC * kEP;
        const R* En = Eb + 3 * eN * kEP;
        R* B1 = Bb + 3 * b1 * kBP;
        // B'(i+1) on rows -1 .. kYTY, z -1 .. kYTZ
        if (warp < kBY && lane < kBZ) {
            const int c = se, jp = c + kEZ, kp = c + 1;
            const int e = sb;
            const R ex = Ec[c], ey = Ec[kEP + c], ez = Ec[2 * kEP + c];
            const R dEz_dy = (Ec[2 * kEP + jp] - ez) * Y.inv[1];
            const R dEy_dz = (Ec[kEP + kp] - ey) * Y.inv[2];
            const R dEx_dz = (Ec[kp] - ex) * Y.inv[2];
            const R dEz_dx = (En[2 * kEP + c] - ez) * Y.inv[0];
            const R dEy_dx = (En[kEP + c] - ey) * Y.inv[0];
            const R dEx_dy = (Ec[jp] - ex) * Y.inv[1];
            const bool out = Y.zopen && !zlo_in;
            B1[e] = out ? R(0) : B1[e] - h * (dEz_dy - dEy_dz);
            B1[kBP + e] = out ? R(0) : B1[kBP + e] - h * (dEx_dz - dEz_dx);
            B1[2 * kBP + e] = out ? R(0) : B1[2 * kBP + e] - h * (dEy_dx - dEx_dy);
        }
        __syncthreads();
        // E'(i+1) on rows 0 .. kYTY, z 0 .. kYTZ (into E(i+1)'s plane)
        if (i >= x0 - 1 && warp < kJY && lane < kJZ) {
            const R* B0 = Bb + 3 * b0 * kBP;
            const R* J1 = Jb + 3 * j1 * kJP;
            R* Ew = Eb + 3 * eC * kEP;
            const int cb = sb + kBZ + 1, jm = cb - kBZ, km = cb - 1;
            const int ce = se + kEZ + 1;
            const int e = sj;
            const R bx_ = B1[cb], by_ = B1[kBP + cb], bz_ = B1[2 * kBP + cb];
            const R dBz_dy = (bz_ - B1[2 * kBP + jm]) * Y.inv[1];
            const R dBy_dz = (by_ - B1[kBP + km]) * Y.inv[2];
            const R dBx_dz = (bx_ - B1[km]) * Y.inv[2];
            const R dBz_dx = (bz_ - B0[2 * kBP + cb]) * Y.inv[0];
            const R dBy_dx = (by_ - B0[kBP + cb]) * Y.inv[0];
            const R dBx_dy = (bx_ - B1[jm]) * Y.inv[1];
            const bool out = Y.zopen && !zj_in;
            Ew[ce] = out ? R(0) : Ew[ce] + Y.dt * ((dBz_dy - dBy_dz) - J1[e]);
            Ew[kEP + ce] = out ? R(0) : Ew[kEP + ce] + Y.dt * ((dBx_dz - dBz_dx) - J1[kJP + e]);
            Ew[2 * kEP + ce] = out ? R(0) : Ew[2 * kEP + ce] + Y.dt * ((dBy_dx - dBx_dy) - J1[2 * kJP + e]);
        }
        __syncthreads();
        // B''(i) on the tile; E'(i) and B''(i) into the other set
        if (i >= x0 && warp < kYTY && lane < kYTZ && j0 + warp < Y.n[1] && zj_in) {
            const R* Ep = Eb + 3 * eP * kEP;
            const R* B0 = Bb + 3 * b0 * kBP;
            const int ce = se + kEZ + 1, jp = ce + kEZ, kp = ce + 1;
            const int cb = sb + kBZ + 1;
            const R ex = Ep[ce], ey = Ep[kEP + ce], ez = Ep[2 * kEP + ce];
            const R dEz_dy = (Ep[2 * kEP + jp] - ez) * Y.inv[1];
            const R dEy_dz = (Ep[kEP + kp] - ey) * Y.inv[2];
            const R dEx_dz = (Ep[kp] - ex) * Y.inv[2];
            const R dEz_dx = (Ec[2 * kEP + ce] - ez) * Y.inv[0];
            const R dEy_dx = (Ec[kEP + ce] - ey) * Y.inv[0];
            const R dEx_dy = (Ep[jp] - ex) * Y.inv[1];
            // the tile's own cells need no wrap: row j0 + warp, z = zj
            const int64_t g = int64_t(i) * sx + int64_t(j0 + warp) * Y.n[2] + zj;
            Y.Bo[0][g] = B0[cb] - h * (dEz_dy - dEy_dz);
            Y.Bo[1][g] = B0[kBP + cb] - h * (dEx_dz - dEz_dx);
            Y.Bo[2][g] = B0[2 * kBP + cb] - h * (dEy_dx - dEx_dy);
            Y.Eo[0][g] = ex;
            Y.Eo[1][g] = ey;
            Y.Eo[2][g] = ez;
        }
        // rotate the rings
        const int ep = eP;
        eP = eC, eC = eN, eN = eL, eL = ep;
        const int bp = b0;
        b0 = b1, b1 = bL, bL = bp;
        const int jq = j1;
        j1 = jL, jL = jq;
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (Y.step && blockIdx.x == 0 && threadIdx.x == 0) *Y.step += 1;
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
    Y.ckc = c->solver;
    return Y;
}

// ---------------------------------------------------------------------------
// particle load / store, field conversion, diagnostics
// ---------------------------------------------------------------------------
template <typename R>
// Particles [base, base + count) from source arrays that start at particle
// `base` (device memory, or pinned host memory the kernel reads directly).
__global__ void k_load(StepArgs<R> A, const double* x, const double* y, const double* z, const double* ux,
                       const double* uy, const double* uz, const double* w, int64_t base, int64_t count, int* id,
                       unsigned long long* wmax) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double wi = i < count ? w[i] : 0.0;
    // largest |w| of the warp (non-negative doubles order like their bit
    // patterns), then one atomic per warp
    unsigned long long wb = 0ull;
    if (i < count && isfinite(wi)) wb = (unsigned long long)__double_as_longlong(fabs(double(R(wi))));
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long other = __shfl_down_sync(0xffffffffu, wb, o);
        wb = other > wb ? other : wb;
    }
    if ((threadIdx.x & 31) == 0 && wb) atomicMax(wmax, wb);
    if (i >= count) return;
    const int64_t p = base + i;
    const Geom& g = A.g;
    const double xs[3] = {x[i], y[i], z[i]};
    const double us[3] = {ux[i], uy[i], uz[i]};
    bool ok = isfinite(wi);
    int cell[3];
    bool gone = false;  // z open: a particle loaded outside [0, Lz) is dropped by the first sort
    for (int a = 0; a < 3; ++a) {
        ok = ok && isfinite(xs[a]) && isfinite(us[a]);
        double xv = isfinite(xs[a]) ? xs[a] : 0.0;
        if (a == 2 && g.zopen && !(xv >= 0.0 && xv < g.L[2])) gone = true, xv = 0.0;
        if (!(xv >= 0.0 && xv < g.L[a])) xv = fmod(xv, g.L[a]);  // fmod is the identity inside [0, L)
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
    A.pa[6][p] = R(wi);
    A.key[p] = gone ? dead_key(g) : key_of(g, cell[0], cell[1], cell[2]);
    id[p] = int(p);
    if (!ok) raise_error(A.err, ERRBIT_PARTICLE);
}

// Particles [p0, p0 + cnt) into element 0.. of the destination arrays.
template <typename R>
__global__ void k_store(StepArgs<R> A, int64_t p0, int64_t cnt, double* x, double* y, double* z, double* ux,
                        double* uy, double* uz, double* w, const int* idsrc, int32_t* id) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int64_t p = p0 + i;
    const Geom& g = A.g;
    double* xs[3] = {x, y, z};
    double* us[3] = {ux, uy, uz};
    int cell[3];
    if (sizeof(R) == 4) cell_of(g, A.key[p], cell[0], cell[1], cell[2]);
    for (int a = 0; a < 3; ++a) {
        if (xs[a]) {
            double v = sizeof(R) == 8 ? double(A.pa[a][p]) : (double(cell[a]) + double(A.pa[a][p])) * g.d[a];
            xs[a][i] = wrap_pos(v, g.L[a]);
        }
        if (us[a]) us[a][i] = double(A.pa[3 + a][p]);
    }
    if (w) w[i] = double(A.pa[6][p]);
    if (id) id[i] = idsrc[p];
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
    // gamma - 1 = |u|^2 / (gamma + 1) (no cancellation for slow particles), per
    // particle in the particles' own precision, summed in FP64
    // FP32: each thread's terms summed in FP32 with Kahan compensation (its
    // few hundred terms then carry about one FP32 rounding), then in FP64.
    R ks = R(0), kc = R(0), ws = R(0), wc = R(0);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < A.np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const R u0 = A.pa[3][p], u1 = A.pa[4][p], u2 = A.pa[5][p], w = A.pa[6][p];
        const R uu = u0 * u0 + u1 * u1 + u2 * u2;
        const R term = w * (uu / (sqrt_<R>(R(1) + uu) + R(1)));
        if (sizeof(R) == 8) {
            ks += term;
            ws += w;
        } else {
            const R y = term - kc, t = ks + y;
            kc = (t - ks) - y;
            ks = t;
            const R y2 = w - wc, t2 = ws + y2;
            wc = (t2 - ws) - y2;
            ws = t2;
        }
    }
    double ke = double(ks) - double(kc), sw = double(ws) - double(wc);
    ke *= m;
    double ch = q * sw;
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

// One warp per z-row (i, j) at a time, its lanes along z.
template <typename R>
__global__ void k_diag_divb(const R* Bx, const R* By, const R* Bz, int nx, int ny, int nz, double dx, double dy,
                            double dz, int zopen, unsigned long long* out) {
    const double ix = 1.0 / dx, iy = 1.0 / dy, iz = 1.0 / dz;
    const int lane = threadIdx.x & 31;
    const int64_t rows = (int64_t)nx * ny;
    double mx = 0.0;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int i = int(r / ny), j = int(r - (int64_t)i * ny);
        const int64_t c0 = r * nz;
        const int64_t ip0 = ((int64_t)wrap_once(i + 1, nx) * ny + j) * nz;
        const int64_t jp0 = ((int64_t)i * ny + wrap_once(j + 1, ny)) * nz;
        for (int k = lane; k < nz; k += 32) {
            const int64_t c = c0 + k;
            const double bz_up = zopen && k + 1 == nz ? 0.0 : double(Bz[c0 + wrap_once(k + 1, nz)]);  // z open: zero beyond the end
            const double v = (double(Bx[ip0 + k]) - double(Bx[c])) * ix + (double(By[jp0 + k]) - double(By[c])) * iy +
                             (bz_up - double(Bz[c])) * iz;
            mx = fmax(mx, fabs(v));
        }
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

// z-rows x chunks of kBlock cells along z
static dim3 yee_grid(const pic_ctx* c) {
    return dim3(unsigned(int64_t(c->g.n[0]) * c->g.n[1]), unsigned((c->g.n[2] + kBlock - 1) / kBlock));
}

cudaError_t launch_yee_b(pic_ctx* c, double h) {
    if (c->prec == PIC_FP64) {
        auto Y = make_yee<double>(c, h);
        if (c->solver) k_yee_b_ckc<double><<<yee_grid(c), kBlock, 0, c->stream>>>(Y);
        else k_yee_b<double><<<yee_grid(c), kBlock, 0, c->stream>>>(Y);
    } else {
        auto Y = make_yee<float>(c, h);
        if (c->solver) k_yee_b_ckc<float><<<yee_grid(c), kBlock, 0, c->stream>>>(Y);
        else k_yee_b<float><<<yee_grid(c), kBlock, 0, c->stream>>>(Y);
    }
    return cudaGetLastError();
}


template <typename R> cudaError_t yee_fused_impl(pic_ctx* c) {
    YeeFusedArgs<R> Y;
    for (int d = 0; d < 3; ++d) {
        Y.E[d] = static_cast<const R*>(c->F[d]);
        Y.B[d] = static_cast<const R*>(c->F[3 + d]);
        Y.J[d] = static_cast<const R*>(c->Fo[6 + d]);
        Y.Eo[d] = static_cast<R*>(c->Fo[d]);
        Y.Bo[d] = static_cast<R*>(c->Fo[3 + d]);
        Y.n[d] = c->g.n[d];
        Y.inv[d] = R(1.0 / c->g.d[d]);
    }
    Y.nt[1] = (c->g.n[1] + kYTY - 1) / kYTY;
    Y.nt[2] = (c->g.n[2] + kYTZ - 1) / kYTZ;
    // x-chunks of 32 cells, halved (down to 8) until the launch fills the GPU
    // about four times over: each chunk pays two partial steps to start
    const int64_t tiles = int64_t(Y.nt[1]) * Y.nt[2];
    const int64_t want = 4 * int64_t(c->sms > 0 ? c->sms : 148) * (c->prec == PIC_FP64 ? 3 : 6);
    Y.xc = 32;
    while (Y.xc > 8 && tiles * ((c->g.n[0] + Y.xc - 1) / Y.xc) < want) Y.xc /= 2;
    Y.nt[0] = (c->g.n[0] + Y.xc - 1) / Y.xc;
    Y.h = R(0.5 * c->dt);
    Y.dt = R(c->dt);
    Y.step = c->d_step;
    Y.zopen = c->g.zopen;
    const int64_t blocks = int64_t(Y.nt[0]) * Y.nt[1] * Y.nt[2];
    k_yee_fused<R><<<unsigned(blocks), kYThreads, yee_fused_smem<R>(), c->stream>>>(Y);
    return cudaGetLastError();
}

cudaError_t launch_yee_fused(pic_ctx* c) {
    return c->prec == PIC_FP64 ? yee_fused_impl<double>(c) : yee_fused_impl<float>(c);
}

// The one-pass update's shared memory can exceed 48 KB (FP64): raised once,
// before any stream capture.
cudaError_t configure_yee_fused() {
    cudaError_t e = cudaFuncSetAttribute(k_yee_fused<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(yee_fused_smem<float>()));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_yee_fused<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(yee_fused_smem<double>()));
    return e;
}

cudaError_t launch_yee_e(pic_ctx* c) {
    if (c->prec == PIC_FP64) {
        auto Y = make_yee<double>(c, c->dt);
        k_yee_e<double><<<yee_grid(c), kBlock, 0, c->stream>>>(Y);
    } else {
        auto Y = make_yee<float>(c, c->dt);
        k_yee_e<float><<<yee_grid(c), kBlock, 0, c->stream>>>(Y);
    }
    return cudaGetLastError();
}

__global__ void k_step_counter(long long* s) { *s += 1; }

cudaError_t launch_step_counter(pic_ctx* c) {
    k_step_counter<<<1, 1, 0, c->stream>>>(c->d_step);
    return cudaGetLastError();
}

cudaError_t launch_load_particles(pic_ctx* c, const double* const src[7], int64_t n, int64_t base) {
    if (n == 0) return cudaSuccess;
    if (c->prec == PIC_FP64) {
        auto A = make_args<double>(c);
        k_load<double><<<blocks_for(n), kBlock, 0, c->stream>>>(A, src[0], src[1], src[2], src[3], src[4], src[5],
                                                               src[6], base, n, c->P[c->cur].id,
                                                               reinterpret_cast<unsigned long long*>(c->err + 6));
    } else {
        auto A = make_args<float>(c);
        k_load<float><<<blocks_for(n), kBlock, 0, c->stream>>>(A, src[0], src[1], src[2], src[3], src[4], src[5],
                                                              src[6], base, n, c->P[c->cur].id,
                                                              reinterpret_cast<unsigned long long*>(c->err + 6));
    }
    return cudaGetLastError();
}

cudaError_t launch_get_particles(pic_ctx* c, double* const dst[7], int32_t* id, int64_t p0, int64_t cnt) {
    if (cnt <= 0) return cudaSuccess;
    if (c->prec == PIC_FP64) {
        auto A = make_args<double>(c);
        k_store<double><<<blocks_for(cnt), kBlock, 0, c->stream>>>(A, p0, cnt, dst[0], dst[1], dst[2], dst[3],
                                                                   dst[4], dst[5], dst[6], c->P[c->cur].id, id);
    } else {
        auto A = make_args<float>(c);
        k_store<float><<<blocks_for(cnt), kBlock, 0, c->stream>>>(A, p0, cnt, dst[0], dst[1], dst[2], dst[3],
                                                                  dst[4], dst[5], dst[6], c->P[c->cur].id, id);
    }
    return cudaGetLastError();
}

cudaError_t launch_field_to_f64(pic_ctx* c, int which, double* dst, int64_t i0, int64_t cnt) {
    if (cnt <= 0) return cudaSuccess;
    if (c->prec == PIC_FP64)
        return cudaMemcpyAsync(dst, static_cast<const double*>(c->F[which]) + i0, cnt * sizeof(double),
                               cudaMemcpyDeviceToDevice, c->stream);
    k_convert<float, double><<<blocks_for(cnt), kBlock, 0, c->stream>>>(
        static_cast<const float*>(c->F[which]) + i0, dst, cnt);
    return cudaGetLastError();
}

cudaError_t launch_field_from_f64(pic_ctx* c, int which, const double* src, int64_t i0, int64_t cnt) {
    if (cnt <= 0) return cudaSuccess;
    if (c->prec == PIC_FP64)
        return cudaMemcpyAsync(static_cast<double*>(c->F[which]) + i0, src, cnt * sizeof(double),
                               cudaMemcpyDeviceToDevice, c->stream);
    k_convert<double, float><<<blocks_for(cnt), kBlock, 0, c->stream>>>(src, static_cast<float*>(c->F[which]) + i0,
                                                                       cnt);
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

// ---------------------------------------------------------------------------
// charge density and the discrete continuity residual (Sec. 3.4.1: the
// Esirkepov current conserves charge exactly; Sec. 2.6 reductions)
// ---------------------------------------------------------------------------
// rho(node) += (q w / dV) S_x S_y S_z of each particle (order-P node weights
// at its position, FP64), periodic fold; with z open nodes beyond the z ends
// take nothing.  One particle per thread, FP64 atomics.
template <int P, typename R> __global__ void __launch_bounds__(kBlock) k_rho(StepArgs<R> A, double q_dv, double* rho) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= A.np) return;
    const Geom& g = A.g;
    int cell[3];
    double f[3];
    if (sizeof(R) == 8) {
#pragma unroll
        for (int a = 0; a < 3; ++a) split_pos(double(A.pa[a][p]), g.d[a], g.n[a], cell[a], f[a]);
    } else {
        const int key = A.key[p];
        if (key < g.kbase || key >= dead_key(g)) return;
        cell_of(g, key, cell[0], cell[1], cell[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) f[a] = double(A.pa[a][p]);
    }
    double w[3][P + 1];
    int first[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) Shape<P, double>::weights(f[a], first[a], w[a]);
    const double qw = q_dv * double(A.pa[6][p]);
#pragma unroll
    for (int i = 0; i <= P; ++i) {
        const int64_t gi = wrap_once(cell[0] + first[0] + i, g.n[0]);
#pragma unroll
        for (int j = 0; j <= P; ++j) {
            const int64_t gj = wrap_once(cell[1] + first[1] + j, g.n[1]);
            const double wij = qw * w[0][i] * w[1][j];
#pragma unroll
            for (int k = 0; k <= P; ++k) {
                const int kz = cell[2] + first[2] + k;
                if (g.zopen && unsigned(kz) >= unsigned(g.n[2])) continue;
                atomicAdd(rho + (gi * g.n[1] + gj) * g.n[2] + wrap_once(kz, g.n[2]), wij * w[2][k]);
            }
        }
    }
}

// r = rho1 - rho0 + dt div J at every node of z-planes [k0, k1), div J the
// nodal divergence of the edge-centred current ((Jx[i] - Jx[i-1])/dx + ...,
// periodic; with z open J beyond the ends is zero); out[0] = max |r|,
// out[1] = max |rho0| (non-negative FP64 values compared as bit patterns).
// One warp per z-row at a time.
template <typename R>
__global__ void k_continuity(const double* rho0, const double* rho1, const R* Jx, const R* Jy, const R* Jz, int nx,
                             int ny, int nz, double dtdx, double dtdy, double dtdz, int zopen, int k0, int k1,
                             unsigned long long* out) {
    const int lane = threadIdx.x & 31;
    const int64_t rows = (int64_t)nx * ny;
    double mr = 0.0, m0 = 0.0;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int i = int(r / ny), j = int(r - (int64_t)i * ny);
        const int64_t c0 = r * nz;
        const int64_t im0 = ((int64_t)wrap_once(i - 1, nx) * ny + j) * nz;
        const int64_t jm0 = ((int64_t)i * ny + wrap_once(j - 1, ny)) * nz;
        for (int k = k0 + lane; k < k1; k += 32) {
            const int64_t c = c0 + k;
            const double jz_dn = zopen && k == 0 ? 0.0 : double(Jz[c0 + wrap_once(k - 1, nz)]);
            const double div = (double(Jx[c]) - double(Jx[im0 + k])) * dtdx +
                               (double(Jy[c]) - double(Jy[jm0 + k])) * dtdy + (double(Jz[c]) - jz_dn) * dtdz;
            const double res = rho1[c] - rho0[c] + div;
            mr = fmax(mr, fabs(res));
            m0 = fmax(m0, fabs(rho0[c]));
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        mr = fmax(mr, __shfl_down_sync(0xffffffffu, mr, o));
        m0 = fmax(m0, __shfl_down_sync(0xffffffffu, m0, o));
    }
    if (lane == 0) {
        atomicMax(out, (unsigned long long)__double_as_longlong(mr));
        atomicMax(out + 1, (unsigned long long)__double_as_longlong(m0));
    }
}

template <typename R, int P> cudaError_t rho_impl(pic_ctx* c, double* rho) {
    k_rho<P, R><<<blocks_for(c->np), kBlock, 0, c->stream>>>(make_args<R>(c),
                                                             c->q / (c->g.d[0] * c->g.d[1] * c->g.d[2]), rho);
    return cudaGetLastError();
}

cudaError_t launch_charge_density(pic_ctx* c, double* rho) {
    cudaError_t e = cudaMemsetAsync(rho, 0, size_t(c->g.C) * sizeof(double), c->stream);
    if (e != cudaSuccess || c->np == 0) return e;
    if (c->prec == PIC_FP64) {
        switch (c->order) {
        case 1: return rho_impl<double, 1>(c, rho);
        case 2: return rho_impl<double, 2>(c, rho);
        default: return rho_impl<double, 3>(c, rho);
        }
    }
    switch (c->order) {
    case 1: return rho_impl<float, 1>(c, rho);
    case 2: return rho_impl<float, 2>(c, rho);
    default: return rho_impl<float, 3>(c, rho);
    }
}

template <typename R>
cudaError_t continuity_impl(pic_ctx* c, const double* rho0, const double* rho1, unsigned long long* out) {
    // with z open the residual covers the planes whose stencils never reach
    // beyond the ends (the current there is dropped, particles leaving are removed)
    const int margin = c->g.zopen ? c->order + 2 : 0;
    const int k0 = margin, k1 = c->g.n[2] - margin;
    const int64_t rows = int64_t(c->g.n[0]) * c->g.n[1];
    const unsigned nb = unsigned(std::min<int64_t>((rows * 32 + kBlock - 1) / kBlock, 152 * 8));
    k_continuity<R><<<nb, kBlock, 0, c->stream>>>(rho0, rho1, static_cast<const R*>(c->F[6]),
                                                  static_cast<const R*>(c->F[7]), static_cast<const R*>(c->F[8]),
                                                  c->g.n[0], c->g.n[1], c->g.n[2], c->dt / c->g.d[0],
                                                  c->dt / c->g.d[1], c->dt / c->g.d[2], c->g.zopen, k0,
                                                  k1 > k0 ? k1 : k0, out);
    return cudaGetLastError();
}

cudaError_t launch_continuity(pic_ctx* c, const double* rho0, const double* rho1, unsigned long long* out) {
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
    return c->prec == PIC_FP64 ? continuity_impl<double>(c, rho0, rho1, out)
                               : continuity_impl<float>(c, rho0, rho1, out);
}

// ---------------------------------------------------------------------------
// z filter of the fields the particles gather (the Godfrey filter of the
// paper's plasma-acceleration run, Sec. 4.2, in its compensated binomial
// form): npass passes of (1/4, 1/2, 1/4) along z, then one compensation pass
// (-npass/4, 1 + npass/2, -npass/4); each pass reads the previous one's output,
// periodic along z or zero beyond the z ends when z is open.  One CTA per z
// column of one component, the column ping-ponging between two shared-memory
// rows of nz values.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kBlock) k_filter_z(const R* __restrict__ F, R* __restrict__ out, int64_t C, int nz,
                                                     int npass, int zopen) {
    extern __shared__ __align__(16) unsigned char filt_raw[];
    R* buf = reinterpret_cast<R*>(filt_raw);  // two rows of nz values
    const int64_t col = blockIdx.x;           // (i ny + j) of the column
    const int comp = blockIdx.y;              // 0..5: Ex..Bz
    const R* src = F + comp * C + col * nz;
    R* dst = out + comp * C + col * nz;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) buf[k] = src[k];
    __syncthreads();
    int cur = 0;
    for (int pass = 0; pass <= npass; ++pass) {
        const R a = pass < npass ? R(0.25) : R(-0.25 * npass);
        const R b = pass < npass ? R(0.5) : R(1.0 + 0.5 * npass);
        const R* in = buf + cur * nz;
        R* o = buf + (1 - cur) * nz;
        for (int k = threadIdx.x; k < nz; k += blockDim.x) {
            const R left = k > 0 ? in[k - 1] : (zopen ? R(0) : in[nz - 1]);
            const R right = k + 1 < nz ? in[k + 1] : (zopen ? R(0) : in[0]);
            o[k] = a * left + b * in[k] + a * right;
        }
        __syncthreads();
        cur = 1 - cur;
    }
    for (int k = threadIdx.x; k < nz; k += blockDim.x) dst[k] = buf[cur * nz + k];
}

size_t filter_smem_bytes(const pic_ctx* c) { return 2 * size_t(c->g.n[2]) * c->rsize; }

cudaError_t configure_filter(const pic_ctx* c) {
    const int bytes = int(filter_smem_bytes(c));
    return c->prec == PIC_FP64
               ? cudaFuncSetAttribute(k_filter_z<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
               : cudaFuncSetAttribute(k_filter_z<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_filter(pic_ctx* c) {
    if (c->filter_passes <= 0 || !c->Fg) return cudaSuccess;
    const dim3 grid(unsigned(int64_t(c->g.n[0]) * c->g.n[1]), 6);
    const size_t smem = filter_smem_bytes(c);
    if (c->prec == PIC_FP64)
        k_filter_z<double><<<grid, kBlock, smem, c->stream>>>(static_cast<const double*>(c->F[0]),
                                                              static_cast<double*>(c->Fg), c->g.C, c->g.n[2],
                                                              c->filter_passes, c->g.zopen);
    else
        k_filter_z<float><<<grid, kBlock, smem, c->stream>>>(static_cast<const float*>(c->F[0]),
                                                             static_cast<float*>(c->Fg), c->g.C, c->g.n[2],
                                                             c->filter_passes, c->g.zopen);
    return cudaGetLastError();
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
