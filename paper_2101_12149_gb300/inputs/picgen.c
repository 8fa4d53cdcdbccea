/*
 * Seeded synthetic particle loading shared by the CUDA library's tests and
 * benchmark and by the CPU oracle's tests.  It holds none of the PIC
 * method's arithmetic: only the counter-based random numbers and the
 * placement recipe of the uniform-plasma workloads.
 *
 * Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator.  For stream key K = splitmix64(seed) and counter
 * c = particle_index * 16 + draw_index, the 64-bit draw is
 * splitmix64(K + c); U[0,1) takes its top 53 bits.  Normals use the
 * cosine branch of Box-Muller: sqrt(-2 ln(1-U1)) cos(2 pi U2).
 *
 * Placement: particles are generated cell-major, then particle-in-cell:
 * particle index = cell * ppc + s with cell = (i*ny + j)*nz + k; position
 * (i + U0, j + U1, k + U2) * d; momentum components u ~ N(0, sigma_u) from
 * draws 3..8; optional x-momentum perturbation amp * sin(kpert * x).
 */
#include <math.h>
#include <stdint.h>

static inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline double unit(uint64_t key, int64_t index, int draw) {
    const uint64_t c = (uint64_t)index * 16u + (uint64_t)draw;
    return (double)(splitmix64(key + c) >> 11) * 0x1.0p-53;
}

static inline double normal(uint64_t key, int64_t index, int draw) {
    const double u1 = unit(key, index, draw), u2 = unit(key, index, draw + 1);
    return sqrt(-2.0 * log(1.0 - u1)) * cos(6.283185307179586476925286766559 * u2);
}

/* U[0,1) draws for counters index in [i0, i0+n), one draw index. */
void pg_uniform(uint64_t seed, int64_t i0, int64_t n, int draw, double* out) {
    const uint64_t key = splitmix64(seed);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < n; ++t) out[t] = unit(key, i0 + t, draw);
}

/* N(0,1) draws (draw, draw+1 consumed) for counters in [i0, i0+n). */
void pg_normal(uint64_t seed, int64_t i0, int64_t n, int draw, double* out) {
    const uint64_t key = splitmix64(seed);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < n; ++t) out[t] = normal(key, i0 + t, draw);
}

/* Uniform plasma, cells [cell0, cell1) of an nx*ny*nz grid, ppc particles
 * per cell; writes (cell1-cell0)*ppc particles starting at out[0]. */
void pg_uniform_plasma(uint64_t seed, int64_t nx, int64_t ny, int64_t nz, int64_t ppc,
                       double dx, double dy, double dz, double sigma_u, double weight,
                       double pert_amp, double pert_k, int64_t cell0, int64_t cell1,
                       double* x, double* y, double* z, double* ux, double* uy, double* uz,
                       double* w) {
    const uint64_t key = splitmix64(seed);
    (void)nx;
#pragma omp parallel for schedule(static)
    for (int64_t c = cell0; c < cell1; ++c) {
        const int64_t i = c / (ny * nz), j = (c / nz) % ny, k = c % nz;
        for (int64_t s = 0; s < ppc; ++s) {
            const int64_t pid = c * ppc + s;
            const int64_t o = (c - cell0) * ppc + s;
            x[o] = ((double)i + unit(key, pid, 0)) * dx;
            y[o] = ((double)j + unit(key, pid, 1)) * dy;
            z[o] = ((double)k + unit(key, pid, 2)) * dz;
            ux[o] = sigma_u * normal(key, pid, 3);
            uy[o] = sigma_u * normal(key, pid, 5);
            uz[o] = sigma_u * normal(key, pid, 7);
            if (pert_amp != 0.0) ux[o] += pert_amp * sin(pert_k * x[o]);
            w[o] = weight;
        }
    }
}
