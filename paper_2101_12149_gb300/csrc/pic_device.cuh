// Device building blocks of the PIC hot path: shape weights, Boris push,
// Esirkepov current weights.  Templated on the arithmetic type R (double for
// the FP64 path, float for FP32-mixed) and the shape order P (1..3).
//
// Positions enter as (integer node, fraction) pairs in cell units, so the
// same code serves the FP64 path (fraction = x/dx - floor(x/dx), exact) and
// the FP32-mixed path (int32 cell + float in-cell offset).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pic_ctx.h"

namespace pic {

__device__ __forceinline__ void raise_error(unsigned* err, unsigned bit) { atomicOr(err, bit); }

__device__ __forceinline__ void check_failed(unsigned* err, unsigned site, long long value) {
    if ((atomicOr(err, ERRBIT_CHECK) & ERRBIT_CHECK) == 0) {
        err[1] = site;
        err[2] = unsigned(value);
        err[3] = unsigned(value >> 32);
    }
}

#ifdef PIC_CHECK
#define PIC_CHECK_OR(cond, err, site, value, action) \
    do {                                            \
        if (!(cond)) {                              \
            ::pic::check_failed(err, site, value);  \
            action;                                 \
        }                                           \
    } while (0)
#else
#define PIC_CHECK_OR(cond, err, site, value, action) \
    do {                                            \
    } while (0)
#endif

__device__ __forceinline__ int wrap_once(int i, int n) {
    // i is within one period of [0, n)
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

__device__ __forceinline__ int wrap_any(int i, int n) {
    // any i, n > 0
    const int r = i % n;
    return r < 0 ? r + n : r;
}

template <typename R> __device__ __forceinline__ R rfloor(R v);
template <> __device__ __forceinline__ double rfloor<double>(double v) { return floor(v); }
template <> __device__ __forceinline__ float rfloor<float>(float v) { return floorf(v); }

template <typename R> __device__ __forceinline__ R sqrt_(R v);
template <> __device__ __forceinline__ double sqrt_<double>(double v) { return sqrt(v); }
template <> __device__ __forceinline__ float sqrt_<float>(float v) { return sqrtf(v); }

// ---------------------------------------------------------------------------
// Order-P cardinal B-spline weights.
//
// A position at node i0 + f (f in [0,1)) has non-zero weights on P+1
// consecutive nodes.  `first` receives the first node relative to i0 and
// w[0..P] the weights s_P(i0 + f - node).  The pieces are the B-spline's
// polynomial pieces written in f.
// ---------------------------------------------------------------------------
template <int P, typename R> struct Shape;

// Order 0 (the unit box on [-1/2, 1/2)): used by the energy-conserving gather at order 1.
template <typename R> struct Shape<0, R> {
    __device__ __forceinline__ static void weights(R f, int& first, R w[1]) {
        first = f >= R(0.5) ? 1 : 0;
        w[0] = R(1);
    }
};

template <typename R> struct Shape<1, R> {
    __device__ __forceinline__ static void weights(R f, int& first, R w[2]) {
        first = 0;
        w[0] = R(1) - f;
        w[1] = f;
    }
};

template <typename R> struct Shape<2, R> {
    __device__ __forceinline__ static void weights(R f, int& first, R w[3]) {
        // nearest node c (0 or 1), g = f - c in [-1/2, 1/2)
        const bool up = f >= R(0.5);
        const R g = up ? f - R(1) : f;
        first = up ? 0 : -1;
        const R a = R(0.5) - g, b = R(0.5) + g;
        w[0] = R(0.5) * a * a;
        w[1] = R(0.75) - g * g;
        w[2] = R(0.5) * b * b;
    }
};

template <typename R> struct Shape<3, R> {
    __device__ __forceinline__ static void weights(R f, int& first, R w[4]) {
        first = -1;
        const R f2 = f * f, f3 = f2 * f;
        const R g = R(1) - f;
        const R sixth = R(1) / R(6);
        w[0] = g * g * g * sixth;
        w[1] = (R(4) - R(6) * f2 + R(3) * f3) * sixth;
        w[2] = (R(1) + R(3) * f + R(3) * f2 - R(3) * f3) * sixth;
        w[3] = f3 * sixth;
    }
};

// Derivatives of the weights with respect to the position (same nodes):
// d/dx s_P(i0 + f - node), piece by piece.
template <int P, typename R> struct ShapeD;

template <typename R> struct ShapeD<1, R> {
    __device__ __forceinline__ static void dweights(R, R d[2]) {
        d[0] = R(-1);
        d[1] = R(1);
    }
};

template <typename R> struct ShapeD<2, R> {
    __device__ __forceinline__ static void dweights(R f, R d[3]) {
        const R g = f >= R(0.5) ? f - R(1) : f;
        d[0] = -(R(0.5) - g);
        d[1] = R(-2) * g;
        d[2] = R(0.5) + g;
    }
};

template <typename R> struct ShapeD<3, R> {
    __device__ __forceinline__ static void dweights(R f, R d[4]) {
        const R g = R(1) - f;
        d[0] = R(-0.5) * g * g;
        d[1] = (R(-2) + R(1.5) * f) * f;
        d[2] = R(0.5) + f - R(1.5) * f * f;
        d[3] = R(0.5) * f * f;
    }
};

template <int P, typename R>
__device__ __forceinline__ void staggered_dweights(R f, R d[P + 1]) {
    const bool hi = f >= R(0.5);
    ShapeD<P, R>::dweights(hi ? f - R(0.5) : f + R(0.5), d);
}

// Weights for a component staggered by half a cell along this axis: the
// position relative to the staggered lattice is (i0 + f) - 1/2.
template <int P, typename R>
__device__ __forceinline__ void staggered_weights(R f, int& first, R w[P + 1]) {
    const bool hi = f >= R(0.5);
    const R g = hi ? f - R(0.5) : f + R(0.5);
    Shape<P, R>::weights(g, first, w);
    if (!hi) first -= 1;
}

// Energy-conserving gather (an option of the paper's plasma-acceleration run,
// Sec. 4.2): along a staggered axis the order drops to P - 1, the order of
// the Esirkepov current along its own direction; the weights fill the first P
// of the P + 1 stencil slots and the last is zero.
template <int P, typename R>
__device__ __forceinline__ void staggered_weights_ec(R f, int& first, R w[P + 1]) {
    R v[P];
    staggered_weights<P - 1, R>(f, first, v);
#pragma unroll
    for (int r = 0; r < P; ++r) w[r] = v[r];
    w[P] = R(0);
}

// ---------------------------------------------------------------------------
// Relativistic Boris push (u = gamma v):
//   k = q dt / (2 m);  u- = u + k E;  g- = sqrt(1 + |u-|^2);  t = k B / g-;
//   s = 2 t / (1 + |t|^2);  u' = u- + u- x t;  u+ = u- + u' x s;  u = u+ + k E.
// The FP32 instantiation pushes a particle whose g-^2 exceeds g2_fp64
// (ultra-relativistic; the library's default threshold is g- > 1e3) wholly in
// FP64: both half kicks, g-, t, s and the rotation, so its stored FP32
// momentum is rounded once per step.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void boris_rotate(R k, const R B[3], R um[3], R gm) {
    const R kg = k / gm;  // one division for the three components of t
    const R t0 = kg * B[0], t1 = kg * B[1], t2 = kg * B[2];
    const R tt = t0 * t0 + t1 * t1 + t2 * t2;
    const R sc = R(2) / (R(1) + tt);
    const R s0 = sc * t0, s1 = sc * t1, s2 = sc * t2;
    const R p0 = um[0] + (um[1] * t2 - um[2] * t1);
    const R p1 = um[1] + (um[2] * t0 - um[0] * t2);
    const R p2 = um[2] + (um[0] * t1 - um[1] * t0);
    um[0] += p1 * s2 - p2 * s1;
    um[1] += p2 * s0 - p0 * s2;
    um[2] += p0 * s1 - p1 * s0;
}

template <typename R>
__device__ __forceinline__ void boris(R k, const R E[3], const R B[3], R u[3], float g2_fp64 = 1e6f) {
    R um[3] = {u[0] + k * E[0], u[1] + k * E[1], u[2] + k * E[2]};
    const R g2 = R(1) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2];
    if (sizeof(R) == 4 && float(g2) > g2_fp64) {
        const double kd = double(k);
        const double Ed[3] = {double(E[0]), double(E[1]), double(E[2])};
        double umd[3] = {double(u[0]) + kd * Ed[0], double(u[1]) + kd * Ed[1], double(u[2]) + kd * Ed[2]};
        const double Bd[3] = {double(B[0]), double(B[1]), double(B[2])};
        const double gmd = sqrt(1.0 + umd[0] * umd[0] + umd[1] * umd[1] + umd[2] * umd[2]);
        boris_rotate<double>(kd, Bd, umd, gmd);
        u[0] = R(umd[0] + kd * Ed[0]);
        u[1] = R(umd[1] + kd * Ed[1]);
        u[2] = R(umd[2] + kd * Ed[2]);
        return;
    }
    boris_rotate<R>(k, B, um, sqrt_<R>(g2));
    u[0] = um[0] + k * E[0];
    u[1] = um[1] + k * E[1];
    u[2] = um[2] + k * E[2];
}

// ---------------------------------------------------------------------------
// Vay's pusher (Vay 2008; an option of the paper's plasma-acceleration run,
// Sec. 4.2): u_new - u = (q dt/m)(E + (v + v_new)/2 x B), solved in closed
// form: u' = u + (q dt/m)(E + v x B / 2), tau = (q dt / 2m) B, u* = u'.tau,
// sigma = 1 + |u'|^2 - |tau|^2, gamma_new^2 = (sigma + sqrt(sigma^2 +
// 4(|tau|^2 + u*^2)))/2, t = tau/gamma_new, s = 1/(1 + |t|^2),
// u_new = s (u' + (u'.t) t + u' x t).  kq = q dt / (2 m).  The FP32
// instantiation pushes wholly in FP64 when |u'|^2 > g2_fp64 (default:
// |u'| > 1e3).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void vay_core(T kq, const T B[3], const T up[3], T u[3]) {
    const T tau[3] = {kq * B[0], kq * B[1], kq * B[2]};
    const T tau2 = tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
    const T ustar = up[0] * tau[0] + up[1] * tau[1] + up[2] * tau[2];
    const T sigma = T(1) + up[0] * up[0] + up[1] * up[1] + up[2] * up[2] - tau2;
    const T gnew = sqrt_<T>(T(0.5) * (sigma + sqrt_<T>(sigma * sigma + T(4) * (tau2 + ustar * ustar))));
    const T t[3] = {tau[0] / gnew, tau[1] / gnew, tau[2] / gnew};
    const T s = T(1) / (T(1) + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    const T ut = up[0] * t[0] + up[1] * t[1] + up[2] * t[2];
    u[0] = s * (up[0] + ut * t[0] + (up[1] * t[2] - up[2] * t[1]));
    u[1] = s * (up[1] + ut * t[1] + (up[2] * t[0] - up[0] * t[2]));
    u[2] = s * (up[2] + ut * t[2] + (up[0] * t[1] - up[1] * t[0]));
}

template <typename R>
__device__ __forceinline__ void vay(R kq, const R E[3], const R B[3], R u[3], float g2_fp64 = 1e6f) {
    const R g0 = sqrt_<R>(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const R v[3] = {u[0] / g0, u[1] / g0, u[2] / g0};
    R up[3];
    up[0] = u[0] + R(2) * kq * E[0] + kq * (v[1] * B[2] - v[2] * B[1]);
    up[1] = u[1] + R(2) * kq * E[1] + kq * (v[2] * B[0] - v[0] * B[2]);
    up[2] = u[2] + R(2) * kq * E[2] + kq * (v[0] * B[1] - v[1] * B[0]);
    if (sizeof(R) == 4 && float(up[0] * up[0] + up[1] * up[1] + up[2] * up[2]) > g2_fp64) {
        // the whole push in FP64 (u' included), rounded once into the FP32 momentum
        const double kd = double(kq);
        const double Bd[3] = {double(B[0]), double(B[1]), double(B[2])};
        const double u0[3] = {double(u[0]), double(u[1]), double(u[2])};
        const double gd = sqrt(1.0 + u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2]);
        const double vd[3] = {u0[0] / gd, u0[1] / gd, u0[2] / gd};
        const double upd[3] = {u0[0] + 2.0 * kd * double(E[0]) + kd * (vd[1] * Bd[2] - vd[2] * Bd[1]),
                               u0[1] + 2.0 * kd * double(E[1]) + kd * (vd[2] * Bd[0] - vd[0] * Bd[2]),
                               u0[2] + 2.0 * kd * double(E[2]) + kd * (vd[0] * Bd[1] - vd[1] * Bd[0])};
        double ud[3];
        vay_core<double>(kd, Bd, upd, ud);
        u[0] = R(ud[0]);
        u[1] = R(ud[1]);
        u[2] = R(ud[2]);
    } else {
        vay_core<R>(kq, B, up, u);
    }
}

// ---------------------------------------------------------------------------
// Esirkepov (2001) weights along one axis.
//
// The particle moves from i0 + f0 to i0 + f1 (cell units, |f1 - f0| < 1).
// The common window of P+2 nodes starts at node i0 + b with
// b = floor(min(f0,f1) - (P+1)/2) + 1, which equals the smaller of the first
// support nodes of the old and the new shape.  b is taken in that second form,
// from the same (node, fraction) split that places the weights: the
// subtraction in the first form rounds for fractions within an ulp of a node
// (FP32 offsets near 1) and would shift the window by one node.  Both shapes
// then start at window slot 0 or 1 and are placed with selects so the arrays
// stay in registers.  S0 / dS hold s_P at the old position and the change
// s_P(new) - s_P(old) on the window.
// ---------------------------------------------------------------------------
template <int P, typename R> struct EsirkAxisD;

template <int P, typename R> struct EsirkAxis {
    static constexpr int NW = P + 2;
    int b;
    bool narrow;  // both shapes start at node b: slot P+1 is zero, and so is the last cumulative sum
    R S0[NW];
    R dS[NW];

    __device__ __forceinline__ void init(R f0, R f1) {
        int first0, first1;
        R w0[P + 1], w1[P + 1];
        Shape<P, R>::weights(f0, first0, w0);
        const R fl1 = rfloor<R>(f1);
        Shape<P, R>::weights(f1 - fl1, first1, w1);
        first1 += int(fl1);
        b = first0 < first1 ? first0 : first1;
        // 0 or 1 each when |f1 - f0| < 1; clamped so a violated precondition
        // cannot index outside the window
        const int off0 = min(first0 - b, 1);
        const int off1 = min(first1 - b, 1);
        narrow = off0 == 0 && off1 == 0;
#pragma unroll
        for (int a = 0; a < NW; ++a) {
            const R s0 = off0 == 0 ? (a <= P ? w0[a] : R(0)) : (a >= 1 ? w0[a - 1] : R(0));
            const R s1 = off1 == 0 ? (a <= P ? w1[a] : R(0)) : (a >= 1 ? w1[a - 1] : R(0));
            S0[a] = s0;
            dS[a] = s1 - s0;
        }
    }
};

// The position derivatives of the old and new shapes on the same window
// (D0[w] = s_P'(x0 - node_w), D1[w] = s_P'(x1 - node_w)), for the adjoint.
template <int P, typename R> struct EsirkAxisD {
    static constexpr int NW = P + 2;
    R D0[NW];
    R D1[NW];

    __device__ __forceinline__ void init(R f0, R f1) {
        int first0, first1;
        R w0[P + 1], w1[P + 1], d0[P + 1], d1[P + 1];
        Shape<P, R>::weights(f0, first0, w0);
        ShapeD<P, R>::dweights(f0, d0);
        const R fl1 = rfloor<R>(f1);
        Shape<P, R>::weights(f1 - fl1, first1, w1);
        ShapeD<P, R>::dweights(f1 - fl1, d1);
        first1 += int(fl1);
        const int b = first0 < first1 ? first0 : first1;
        const int off0 = min(first0 - b, 1);
        const int off1 = min(first1 - b, 1);
#pragma unroll
        for (int a = 0; a < NW; ++a) {
            D0[a] = off0 == 0 ? (a <= P ? d0[a] : R(0)) : (a >= 1 ? d0[a - 1] : R(0));
            D1[a] = off1 == 0 ? (a <= P ? d1[a] : R(0)) : (a >= 1 ? d1[a - 1] : R(0));
        }
    }
};

}  // namespace pic
