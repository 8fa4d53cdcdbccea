// Adjoint kernels of libpic: the discrete adjoint of one PIC step (the
// differentiation workload's pic_step_adjoint).  Reverse order of the step:
//   k_adj_yee_e / k_adj_yee_b   transposed Yee update (the two discrete curls
//                               are each other's transposes on the periodic
//                               grid), producing the adjoint of J;
//   k_adj_particles             per particle: recompute gather, Boris and
//                               advance from the stored state, then the
//                               adjoints of the Esirkepov deposit, the
//                               advance, the Boris rotation, the drive and
//                               the gather (a scatter into the field
//                               adjoints).
// Particle adjoints are indexed by particle id, so the sorts between steps
// need no reverse pass.  Cell indices and Esirkepov windows are held fixed
// (the derivative of floor() is zero); the periodic wrap is the identity.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "pic_ctx.h"
#include "pic_device.cuh"
#include "pic_step_common.cuh"

namespace pic {

constexpr int kAdjBlock = 256;

template <typename R> struct AdjArgs {
    R* lamx[3];        // adjoint of the position (cell units), by particle id
    R* lamu[3];        // adjoint of the momentum, by particle id
    R* lamE[3];
    R* lamB[3];
    const R* lamJ[3];
    const int* id;     // ids of the stored particle state
    double* lamA;      // adjoint of the drive amplitude (accumulated)
    double t;          // time of the step's gather
};

// Reverse sweep of the Boris rotation (boris() in pic_device.cuh): given the
// forward inputs and the adjoint of the new momentum, the adjoints of the old
// momentum, of E and of B at the particle.
template <typename R>
__device__ __forceinline__ void boris_adj(R k, const R E[3], const R B[3], const R u_old[3], const R lam_new[3],
                                          R lam_old[3], R lE[3], R lB[3]) {
    R um[3], t[3], s[3], up[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) um[a] = u_old[a] + k * E[a];
    const R gm = sqrt_<R>(R(1) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) t[a] = k * B[a] / gm;
    const R tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    const R sc = R(2) / (R(1) + tt);
#pragma unroll
    for (int a = 0; a < 3; ++a) s[a] = sc * t[a];
    up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    const R* g = lam_new;
    R g_um[3], g_up[3], g_s[3], g_t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lE[a] = k * g[a];
        g_um[a] = g[a];
    }
    // u_new = um + up x s + k E
    g_up[0] = s[1] * g[2] - s[2] * g[1];
    g_up[1] = s[2] * g[0] - s[0] * g[2];
    g_up[2] = s[0] * g[1] - s[1] * g[0];
    g_s[0] = g[1] * up[2] - g[2] * up[1];
    g_s[1] = g[2] * up[0] - g[0] * up[2];
    g_s[2] = g[0] * up[1] - g[1] * up[0];
    // up = um + um x t
    g_um[0] += g_up[0] + (t[1] * g_up[2] - t[2] * g_up[1]);
    g_um[1] += g_up[1] + (t[2] * g_up[0] - t[0] * g_up[2]);
    g_um[2] += g_up[2] + (t[0] * g_up[1] - t[1] * g_up[0]);
    g_t[0] = g_up[1] * um[2] - g_up[2] * um[1];
    g_t[1] = g_up[2] * um[0] - g_up[0] * um[2];
    g_t[2] = g_up[0] * um[1] - g_up[1] * um[0];
    // s = sc t, sc = 2 / (1 + |t|^2)
    R g_sc = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g_t[a] += sc * g_s[a];
        g_sc += g_s[a] * t[a];
    }
    const R g_tt = R(-0.5) * sc * sc * g_sc;
    R g_gm = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g_t[a] += R(2) * t[a] * g_tt;
        lB[a] = (k / gm) * g_t[a];
        g_gm -= t[a] * g_t[a] / gm;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g_um[a] += um[a] / gm * g_gm;
        lam_old[a] = g_um[a];
        lE[a] += k * g_um[a];
    }
}

// Adjoint of the Esirkepov current of component C (cumulative along C,
// transverse T1, T2): J_C(w0,w1,w2) = coef * cum_C(w0) * Q(w1,w2), with
// Q = S0a S0b + dSa S0b/2 + S0a dSb/2 + dSa dSb/3.  Accumulates dL/dS0 and
// dL/ddS per axis; nodes are the window's wrapped element offsets per axis.
template <int P, typename R, int C>
__device__ __forceinline__ void esirkepov_adj_component(const EsirkAxis<P, R>* ax, const int (*node)[P + 2],
                                                        const R* __restrict__ lamJ, R coef, R (*gS0)[P + 2],
                                                        R (*gdS)[P + 2]) {
    constexpr int NW = P + 2;
    constexpr int T1 = (C + 1) % 3, T2 = (C + 2) % 3;
    R cum[NW - 1], gcum[NW - 1];
    R run = R(0);
#pragma unroll
    for (int w = 0; w < NW - 1; ++w) {
        run += ax[C].dS[w];
        cum[w] = run;
        gcum[w] = R(0);
    }
#pragma unroll
    for (int w1 = 0; w1 < NW; ++w1)
#pragma unroll
        for (int w2 = 0; w2 < NW; ++w2) {
            const R S0a = ax[T1].S0[w1], dSa = ax[T1].dS[w1];
            const R S0b = ax[T2].S0[w2], dSb = ax[T2].dS[w2];
            const R Q = S0a * S0b + R(0.5) * dSa * S0b + R(0.5) * S0a * dSb + R(1.0 / 3.0) * dSa * dSb;
            R gQ = R(0);
#pragma unroll
            for (int w0 = 0; w0 < NW - 1; ++w0) {
                const R M = coef * lamJ[node[C][w0] + node[T1][w1] + node[T2][w2]];
                gQ += M * cum[w0];
                gcum[w0] += M * Q;
            }
            gS0[T1][w1] += gQ * (S0b + R(0.5) * dSb);
            gdS[T1][w1] += gQ * (R(0.5) * S0b + R(1.0 / 3.0) * dSb);
            gS0[T2][w2] += gQ * (S0a + R(0.5) * dSa);
            gdS[T2][w2] += gQ * (R(0.5) * S0a + R(1.0 / 3.0) * dSa);
        }
    // cum(w) = sum_{v <= w} dS(v): dL/ddS(v) = sum_{w >= v} dL/dcum(w)
    R acc = R(0);
#pragma unroll
    for (int w = NW - 2; w >= 0; --w) {
        acc += gcum[w];
        gdS[C][w] += acc;
    }
}

// Adjoint of the gather of one field component with staggering (SX, SY, SZ):
// lamF(node) += w(node) lam, and lx += lam * dF/dx (cell units).
template <int P, typename R, bool SX, bool SY, bool SZ>
__device__ __forceinline__ void gather_adj_component(const GatherW<P, R>& G, const R (*dn)[P + 1],
                                                     const R (*ds)[P + 1], const R* __restrict__ F, R* lF, R lam,
                                                     R lx[3]) {
    R g0 = R(0), g1 = R(0), g2 = R(0);
#pragma unroll
    for (int i = 0; i <= P; ++i) {
        const R wx = SX ? G.ws[0][i] : G.wn[0][i];
        const R dwx = SX ? ds[0][i] : dn[0][i];
        const int ox = SX ? G.os[0][i] : G.on[0][i];
#pragma unroll
        for (int j = 0; j <= P; ++j) {
            const R wy = SY ? G.ws[1][j] : G.wn[1][j];
            const R dwy = SY ? ds[1][j] : dn[1][j];
            const int oy = SY ? G.os[1][j] : G.on[1][j];
            R a0 = R(0), a1 = R(0), a2 = R(0);
#pragma unroll
            for (int k = 0; k <= P; ++k) {
                const R wz = SZ ? G.ws[2][k] : G.wn[2][k];
                const R dwz = SZ ? ds[2][k] : dn[2][k];
                const int o = ox + oy + (SZ ? G.os[2][k] : G.on[2][k]);
                const R f = F[o];
                atomicAdd(lF + o, wx * wy * wz * lam);
                a0 += wz * f;
                a2 += dwz * f;
            }
            g0 += dwx * wy * a0;
            g1 += wx * dwy * a0;
            g2 += wx * wy * a2;
            (void)a1;
        }
    }
    lx[0] += lam * g0;
    lx[1] += lam * g1;
    lx[2] += lam * g2;
}

template <int P, typename R>
__global__ void __launch_bounds__(kAdjBlock) k_adj_particles(StepArgs<R> A, AdjArgs<R> L) {
    constexpr int NW = P + 2;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double lamA = 0.0;
    if (p < A.np) {
        const Geom& g = A.g;
        int cell[3];
        R f0[3], u_old[3], wq;
        double xg0[3];
        load_particle<R>(A, int(p), cell, f0, xg0, u_old, wq);
        const int id = L.id[p];
        // ---- forward recomputation ----------------------------------
        GatherW<P, R> G;
        int fn[3], fs[3];
        gather_weights<P, R>(f0, G, fn, fs);
        offsets_global<P, R>(G, g, cell, fn, fs);
        R EB[6];
        gather6<P, R>(G, A.E, A.B, EB);
        double phase = 0.0;
        if (A.drive_amp != 0.0) {
            const double xp = sizeof(R) == 8 ? xg0[0] : (double(cell[0]) + double(f0[0])) * g.d[0];
            phase = A.drive_k * xp - A.drive_k * L.t;
            EB[1] += R(A.drive_amp * cos(phase));
        }
        R u[3] = {u_old[0], u_old[1], u_old[2]};
        Moved<R> mv;
        {
            StepArgs<R> A0 = A;
            A0.drive_amp = 0.0;  // already added above, at the step's own time
            R EBc[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) EBc[c] = EB[c];
            push_particle<P, R>(A0, EBc, cell, f0, xg0, u, mv);
        }
        // ---- adjoints of the step's outputs --------------------------
        R lx1[3], lu[3], lx0[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lx1[a] = L.lamx[a][id];
            lu[a] = L.lamu[a][id];
        }
        // ---- Esirkepov deposit -------------------------------------------
        {
            EsirkAxis<P, R> ax[3];
            int node[3][NW];
            const int st[3] = {g.n[1] * g.n[2], g.n[2], 1};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                ax[a].init(mv.f0[a], mv.f1[a]);
#pragma unroll
                for (int w = 0; w < NW; ++w) node[a][w] = wrap_once(cell[a] + ax[a].b + w, g.n[a]) * st[a];
            }
            R gS0[3][NW], gdS[3][NW];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int w = 0; w < NW; ++w) gS0[a][w] = gdS[a][w] = R(0);
            esirkepov_adj_component<P, R, 0>(ax, node, L.lamJ[0], A.jc[0] * wq, gS0, gdS);
            esirkepov_adj_component<P, R, 1>(ax, node, L.lamJ[1], A.jc[1] * wq, gS0, gdS);
            esirkepov_adj_component<P, R, 2>(ax, node, L.lamJ[2], A.jc[2] * wq, gS0, gdS);
            // dS = S1 - S0: dL/dS1 = gdS, dL/dS0 = gS0 - gdS; then the chain
            // through the shape derivatives on the same window
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                EsirkAxisD<P, R> dx;
                dx.init(mv.f0[a], mv.f1[a]);
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    lx0[a] += (gS0[a][w] - gdS[a][w]) * dx.D0[w];
                    lx1[a] += gdS[a][w] * dx.D1[w];
                }
            }
        }
        // ---- advance: f1 = f0 + (dt/d) u / gamma ------------------------
        {
            const R gam = sqrt_<R>(R(1) + mv.u[0] * mv.u[0] + mv.u[1] * mv.u[1] + mv.u[2] * mv.u[2]);
            R sdot = R(0);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lx0[a] += lx1[a];
                sdot += A.dtc[a] * lx1[a] * mv.u[a];
            }
            const R g3 = gam * gam * gam;
#pragma unroll
            for (int a = 0; a < 3; ++a) lu[a] += A.dtc[a] * lx1[a] / gam - mv.u[a] * sdot / g3;
        }
        // ---- Boris ----------------------------------------------------
        R luo[3], lE[3], lB[3];
        boris_adj<R>(A.kq, EB, EB + 3, u_old, lu, luo, lE, lB);
        // ---- drive ------------------------------------------------------
        if (A.drive_amp != 0.0) {
            lamA += double(lE[1]) * cos(phase);
            lx0[0] += R(double(lE[1]) * A.drive_amp * (-A.drive_k) * sin(phase) * g.d[0]);
        }
        // ---- gather ----------------------------------------------------
        {
            R dn[3][P + 1], ds[3][P + 1];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                ShapeD<P, R>::dweights(f0[a], dn[a]);
                staggered_dweights<P, R>(f0[a], ds[a]);
            }
            // staggering along x, y, z: Ex (s,n,n) Ey (n,s,n) Ez (n,n,s) Bx (n,s,s) By (s,n,s) Bz (s,s,n)
            gather_adj_component<P, R, true, false, false>(G, dn, ds, A.E[0], L.lamE[0], lE[0], lx0);
            gather_adj_component<P, R, false, true, false>(G, dn, ds, A.E[1], L.lamE[1], lE[1], lx0);
            gather_adj_component<P, R, false, false, true>(G, dn, ds, A.E[2], L.lamE[2], lE[2], lx0);
            gather_adj_component<P, R, false, true, true>(G, dn, ds, A.B[0], L.lamB[0], lB[0], lx0);
            gather_adj_component<P, R, true, false, true>(G, dn, ds, A.B[1], L.lamB[1], lB[1], lx0);
            gather_adj_component<P, R, true, true, false>(G, dn, ds, A.B[2], L.lamB[2], lB[2], lx0);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            L.lamx[a][id] = lx0[a];
            L.lamu[a][id] = luo[a];
        }
    }
    // block sum of the drive adjoint
    for (int o = 16; o; o >>= 1) lamA += __shfl_down_sync(0xffffffffu, lamA, o);
    __shared__ double red[kAdjBlock / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lamA;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kAdjBlock / 32; ++w) s += red[w];
        if (s != 0.0) atomicAdd(L.lamA, s);
    }
}

// lamE -= h curl' lamB (backward-difference curl, the transpose of the curl in
// the B update).
template <typename R>
__global__ void __launch_bounds__(kAdjBlock) k_adj_yee_e(R* lE0, R* lE1, R* lE2, const R* lB0, const R* lB1,
                                                         const R* lB2, int nx, int ny, int nz, R ix, R iy, R iz, R h) {
    const int64_t C = (int64_t)nx * ny * nz;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int k = int(c % nz), j = int((c / nz) % ny), i = int(c / ((int64_t)ny * nz));
    const int64_t sx = (int64_t)ny * nz, sy = nz;
    const int64_t im = c - (i == 0 ? -(int64_t)(nx - 1) * sx : sx);
    const int64_t jm = c - (j == 0 ? -(int64_t)(ny - 1) * sy : sy);
    const int64_t km = c - (k == 0 ? -(int64_t)(nz - 1) : 1);
    const R bx = lB0[c], by = lB1[c], bz = lB2[c];
    lE0[c] -= h * ((bz - lB2[jm]) * iy - (by - lB1[km]) * iz);
    lE1[c] -= h * ((bx - lB0[km]) * iz - (bz - lB2[im]) * ix);
    lE2[c] -= h * ((by - lB1[im]) * ix - (bx - lB0[jm]) * iy);
}

// lamJ = -dt lamE; lamB += dt curl lamE (forward-difference curl, the
// transpose of the curl in the E update).
template <typename R>
__global__ void __launch_bounds__(kAdjBlock) k_adj_yee_b(const R* lE0, const R* lE1, const R* lE2, R* lB0, R* lB1,
                                                         R* lB2, R* lJ0, R* lJ1, R* lJ2, int nx, int ny, int nz, R ix,
                                                         R iy, R iz, R dt) {
    const int64_t C = (int64_t)nx * ny * nz;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int k = int(c % nz), j = int((c / nz) % ny), i = int(c / ((int64_t)ny * nz));
    const int64_t sx = (int64_t)ny * nz, sy = nz;
    const int64_t ip = c + (i + 1 == nx ? -(int64_t)(nx - 1) * sx : sx);
    const int64_t jp = c + (j + 1 == ny ? -(int64_t)(ny - 1) * sy : sy);
    const int64_t kp = c + (k + 1 == nz ? -(int64_t)(nz - 1) : 1);
    const R ex = lE0[c], ey = lE1[c], ez = lE2[c];
    lJ0[c] = -dt * ex;
    lJ1[c] = -dt * ey;
    lJ2[c] = -dt * ez;
    lB0[c] += dt * ((lE2[jp] - ez) * iy - (lE1[kp] - ey) * iz);
    lB1[c] += dt * ((lE0[kp] - ex) * iz - (lE2[ip] - ez) * ix);
    lB2[c] += dt * ((lE1[ip] - ey) * ix - (lE0[jp] - ex) * iy);
}

// Reverse of one Yee step (B half, E full, B half):
//   lamE -= h C^T lamB;  lamJ = -dt lamE, lamB += dt C'^T lamE;  lamE -= h C^T lamB.
template <typename R> cudaError_t adj_yee_impl(pic_ctx* c, const AdjBuffers& b) {
    const int nx = c->g.n[0], ny = c->g.n[1], nz = c->g.n[2];
    const unsigned nb = unsigned((c->g.C + kAdjBlock - 1) / kAdjBlock);
    R* lE[3];
    R* lB[3];
    R* lJ[3];
    for (int a = 0; a < 3; ++a) {
        lE[a] = static_cast<R*>(b.lamE[a]);
        lB[a] = static_cast<R*>(b.lamB[a]);
        lJ[a] = static_cast<R*>(b.lamJ[a]);
    }
    const R ix = R(1.0 / c->g.d[0]), iy = R(1.0 / c->g.d[1]), iz = R(1.0 / c->g.d[2]);
    const R h = R(0.5 * c->dt), dt = R(c->dt);
    k_adj_yee_e<R><<<nb, kAdjBlock, 0, c->stream>>>(lE[0], lE[1], lE[2], lB[0], lB[1], lB[2], nx, ny, nz, ix, iy, iz, h);
    k_adj_yee_b<R><<<nb, kAdjBlock, 0, c->stream>>>(lE[0], lE[1], lE[2], lB[0], lB[1], lB[2], lJ[0], lJ[1], lJ[2], nx,
                                                    ny, nz, ix, iy, iz, dt);
    k_adj_yee_e<R><<<nb, kAdjBlock, 0, c->stream>>>(lE[0], lE[1], lE[2], lB[0], lB[1], lB[2], nx, ny, nz, ix, iy, iz, h);
    return cudaGetLastError();
}

cudaError_t launch_adj_yee(pic_ctx* c, const AdjBuffers& b) {
    return c->prec == PIC_FP64 ? adj_yee_impl<double>(c, b) : adj_yee_impl<float>(c, b);
}

template <typename R, int P> cudaError_t adj_particles_impl(pic_ctx* c, const AdjBuffers& b, const Snapshot& s,
                                                           double t) {
    StepArgs<R> A = make_args<R>(c);
    // the stored state replaces the live particles and fields
    for (int i = 0; i < 7; ++i) {
        A.pa[i] = static_cast<R*>(s.a[i]);
        A.spa[i] = A.pa[i];
    }
    A.key = s.key;
    A.skey = s.key;
    A.sid = A.did = s.id;
    for (int d = 0; d < 3; ++d) {
        A.E[d] = static_cast<const R*>(s.F[d]);
        A.B[d] = static_cast<const R*>(s.F[3 + d]);
    }
    AdjArgs<R> L;
    for (int a = 0; a < 3; ++a) {
        L.lamx[a] = static_cast<R*>(b.lamx[a]);
        L.lamu[a] = static_cast<R*>(b.lamu[a]);
        L.lamE[a] = static_cast<R*>(b.lamE[a]);
        L.lamB[a] = static_cast<R*>(b.lamB[a]);
        L.lamJ[a] = static_cast<const R*>(b.lamJ[a]);
    }
    L.id = s.id;
    L.lamA = b.lamA;
    L.t = t;
    if (c->np == 0) return cudaSuccess;
    k_adj_particles<P, R><<<unsigned((c->np + kAdjBlock - 1) / kAdjBlock), kAdjBlock, 0, c->stream>>>(A, L);
    return cudaGetLastError();
}

cudaError_t launch_adj_particles(pic_ctx* c, const AdjBuffers& b, const Snapshot& s, double t) {
    if (c->prec == PIC_FP64) {
        switch (c->order) {
        case 1: return adj_particles_impl<double, 1>(c, b, s, t);
        case 2: return adj_particles_impl<double, 2>(c, b, s, t);
        default: return adj_particles_impl<double, 3>(c, b, s, t);
        }
    }
    switch (c->order) {
    case 1: return adj_particles_impl<float, 1>(c, b, s, t);
    case 2: return adj_particles_impl<float, 2>(c, b, s, t);
    default: return adj_particles_impl<float, 3>(c, b, s, t);
    }
}

template <typename S, typename D> __global__ void k_copy_convert(const S* src, D* dst, int64_t n, D scale) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = D(src[i]) * scale;
}

// lamE = E dV, lamB = B dV (adjoint of L = 1/2 sum |E|^2 + |B|^2 dV); zero the rest.
cudaError_t launch_adj_init(pic_ctx* c, const AdjBuffers& b) {
    const unsigned nb = unsigned((c->g.C + kAdjBlock - 1) / kAdjBlock);
    const double dV = c->g.d[0] * c->g.d[1] * c->g.d[2];
    for (int a = 0; a < 3; ++a) {
        if (c->prec == PIC_FP64) {
            k_copy_convert<double, double><<<nb, kAdjBlock, 0, c->stream>>>(
                static_cast<const double*>(c->F[a]), static_cast<double*>(b.lamE[a]), c->g.C, dV);
            k_copy_convert<double, double><<<nb, kAdjBlock, 0, c->stream>>>(
                static_cast<const double*>(c->F[3 + a]), static_cast<double*>(b.lamB[a]), c->g.C, dV);
        } else {
            k_copy_convert<float, float><<<nb, kAdjBlock, 0, c->stream>>>(
                static_cast<const float*>(c->F[a]), static_cast<float*>(b.lamE[a]), c->g.C, float(dV));
            k_copy_convert<float, float><<<nb, kAdjBlock, 0, c->stream>>>(
                static_cast<const float*>(c->F[3 + a]), static_cast<float*>(b.lamB[a]), c->g.C, float(dV));
        }
    }
    return cudaGetLastError();
}

// dL/du (by id, component-major, FP64) from the momentum adjoint.
cudaError_t launch_adj_output(pic_ctx* c, const AdjBuffers& b, double* d_out) {
    if (c->np == 0) return cudaSuccess;
    const unsigned nb = unsigned((c->np + kAdjBlock - 1) / kAdjBlock);
    for (int a = 0; a < 3; ++a) {
        if (c->prec == PIC_FP64)
            k_copy_convert<double, double><<<nb, kAdjBlock, 0, c->stream>>>(static_cast<const double*>(b.lamu[a]),
                                                                            d_out + a * c->np, c->np, 1.0);
        else
            k_copy_convert<float, double><<<nb, kAdjBlock, 0, c->stream>>>(static_cast<const float*>(b.lamu[a]),
                                                                           d_out + a * c->np, c->np, 1.0);
    }
    return cudaGetLastError();
}

}  // namespace pic
