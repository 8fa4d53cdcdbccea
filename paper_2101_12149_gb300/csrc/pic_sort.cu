// Counting sort of the particles by tile-major cell key (Sec. 3.4.2: bin by
// cell, then reorder the particle data; AMReX builds its GPU counting sort on
// the single-pass prefix sum of Merrill and Garland).
//
//  k_hist     count[key] += 1, one atomic per run of equal keys in a warp
//  k_scan     exclusive prefix sum of count into offsets in one pass:
//             each CTA takes the next chunk ticket, publishes its aggregate,
//             and looks back over its predecessors' published words
//             (decoupled look-back, Merrill & Garland 2016).  Every wait is
//             bounded; a wait that runs out sets the device error word.
//  k_scatter  each particle takes a slot in its cell's range by decrementing
//             count (one atomic per run of equal keys), then all its arrays move to the other
//             buffer.  count returns to zero, ready for the next histogram.
//  k_bin_keys pic_sort_particles only: coarse (runs of cells) or random bins
//             for the same three kernels; the cell key moves as data.
#include <cuda_runtime.h>

#include <cstdint>

#include "pic_ctx.h"
#include "pic_device.cuh"
#include "pic_sort.cuh"

namespace pic {

constexpr int kSpinLimit = 1 << 20;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// The lanes of this lane's run of equal keys among consecutive lanes.  The
// particles are mostly in cell order already (sorted the step before), so a
// run is usually all of a key's lanes; a key split over several runs just
// takes one atomic per run.  Cheaper than __match_any_sync.
__device__ __forceinline__ unsigned run_mask(int k) {
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(0xffffffffu, k, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != k);
    const unsigned upto = (2u << lane) - 1u;  // lanes <= lane (all for lane 31)
    const int first = 31 - __clz(heads & upto);
    const unsigned above = heads & ~upto;
    const unsigned below_end = above ? (1u << (__ffs(above) - 1)) - 1u : 0xffffffffu;
    return below_end & ~((1u << first) - 1u);
}

__global__ void __launch_bounds__(kSortBlock) k_hist(const int* __restrict__ key, int64_t np, int* count, int64_t C,
                                                     unsigned* err) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int k = -1;
    if (p < np) {
        k = key[p];
        if (k < 0 || k >= C) {
            raise_error(err, ERRBIT_RANGE);
            k = -1;
        }
    }
    const unsigned mask = run_mask(k);
    if (k >= 0) {
        const int lane = threadIdx.x & 31;
        if (lane == __ffs(mask) - 1) atomicAdd(count + k, __popc(mask));
    }
}

// status word: bits 32..33 flag (0 empty, 1 aggregate, 2 inclusive prefix), low 32 bits value
__device__ __forceinline__ unsigned long long ld_status(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_status(unsigned long long* p, unsigned flag, unsigned value) {
    const unsigned long long v = ((unsigned long long)flag << 32) | value;
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__global__ void __launch_bounds__(kSortBlock) k_scan(const int* __restrict__ count, int* offsets, int64_t C,
                                                     unsigned long long* status, int nchunks, unsigned* err) {
    __shared__ int s_chunk;
    __shared__ int s_warp[kSortBlock / 32];
    __shared__ int s_prefix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_chunk = int(atomicAdd(reinterpret_cast<unsigned long long*>(status + nchunks), 1ull));
    __syncthreads();
    const int chunk = s_chunk;
    if (chunk >= nchunks) return;
    const int64_t base = (int64_t)chunk * kScanChunk + (int64_t)tid * kScanItems;

    // a thread's kScanItems consecutive counts: four 16-byte loads when the
    // group lies inside [0, C) and the arrays are 16-byte aligned (always for
    // the library's own arrays), else one count at a time
    const bool vec = base + kScanItems <= C &&
                     ((reinterpret_cast<uintptr_t>(count) | reinterpret_cast<uintptr_t>(offsets)) & 15) == 0;
    int v[kScanItems];
    int tsum = 0;
    if (vec) {
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            const int4 c4 = reinterpret_cast<const int4*>(count + base)[q];
            v[4 * q] = c4.x, v[4 * q + 1] = c4.y, v[4 * q + 2] = c4.z, v[4 * q + 3] = c4.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const int64_t idx = base + i;
            v[i] = idx < C ? count[idx] : 0;
        }
    }
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) tsum += v[i];
    // block exclusive scan of the per-thread sums
    int incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int wv = lane < kSortBlock / 32 ? s_warp[lane] : 0;
        int wi = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kSortBlock / 32) s_warp[lane] = wi - wv;  // exclusive warp offsets
        // the chunk aggregate is the last inclusive value
        const int agg = __shfl_sync(0xffffffffu, wi, kSortBlock / 32 - 1);
        // decoupled look-back by warp 0
        int excl = 0;
        if (chunk == 0) {
            if (lane == 0) st_status(status + chunk, 2u, unsigned(agg));
        } else {
            if (lane == 0) st_status(status + chunk, 1u, unsigned(agg));
            int j = chunk - 1;  // highest predecessor not yet summed
            bool done = false;
            while (!done) {
                const int idx = j - lane;
                unsigned long long s = 0;
                if (idx >= 0) {
                    int spins = 0;
                    s = ld_status(status + idx);
                    while ((s >> 32) == 0ull) {
                        if (++spins > kSpinLimit) {
                            raise_error(err, ERRBIT_TIMEOUT);
                            s = 2ull << 32;  // give up: treat as a zero prefix
                            break;
                        }
                        __nanosleep(32);
                        s = ld_status(status + idx);
                    }
                } else {
                    s = 2ull << 32;  // before chunk 0: empty prefix
                }
                const unsigned flag = unsigned(s >> 32);
                const unsigned incl_mask = __ballot_sync(0xffffffffu, flag == 2u);
                // lanes up to and including the nearest inclusive word contribute
                const int stop = incl_mask ? __ffs(incl_mask) - 1 : 31;
                int contrib = lane <= stop ? int(unsigned(s)) : 0;
#pragma unroll
                for (int o = 16; o; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
                excl += contrib;
                if (incl_mask) done = true;
                else j -= 32;
            }
            if (lane == 0) st_status(status + chunk, 2u, unsigned(excl + agg));
        }
        if (lane == 0) {
            s_prefix = excl;
            if (chunk == nchunks - 1) offsets[C] = excl + agg;
        }
    }
    __syncthreads();
    int run = s_prefix + s_warp[warp] + (incl - tsum);
    PIC_CHECK_OR(run >= 0, err, 7, run, run = 0);
    if (vec) {
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            int4 o;
            o.x = run;
            o.y = o.x + v[4 * q];
            o.z = o.y + v[4 * q + 1];
            o.w = o.z + v[4 * q + 2];
            run = o.w + v[4 * q + 3];
            reinterpret_cast<int4*>(offsets + base)[q] = o;
        }
    } else {
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const int64_t idx = base + i;
            if (idx < C) offsets[idx] = run;
            run += v[i];
        }
    }
}

// `bin` is the array of sort bins: the cell keys themselves (the step's
// sort) or the bins of pic_sort_particles; the cell key always moves with
// the particle.
template <typename E>
__global__ void __launch_bounds__(kSortBlock) k_scatter(PartBuf src, PartBuf dst, const int* __restrict__ bin,
                                                        int64_t np, const int* offsets, int* count, int64_t C,
                                                        unsigned* err) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int k = -1, key = 0;
    // the particle's data is loaded first: these loads do not depend on the
    // slot, so their latency overlaps the atomic that finds it
    E v[7];
    int id = 0;
    if (p < np) {
        k = bin[p];
        key = bin == src.key ? k : src.key[p];
        if (k < 0 || k >= C) k = -1;
#pragma unroll
        for (int i = 0; i < 7; ++i) v[i] = static_cast<const E*>(src.a[i])[p];
        id = src.id[p];
    }
    const int base = k >= 0 ? offsets[k] : 0;  // loaded before the atomic, as in k_scatter_perm
    const unsigned mask = run_mask(k);
    if (k < 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    const int ng = __popc(mask);
    int old = 0;
    if (lane == leader) old = atomicSub(count + k, ng);
    old = __shfl_sync(mask, old, leader);
    const int dest = base + (old - ng) + __popc(mask & lanemask_lt());
    // checked in every build: a histogram that does not match the keys
    // (a step stopped part-way) must not send a particle outside the arrays
    if (!(dest >= 0 && dest < np)) {
        check_failed(err, 8, dest);
        return;
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) static_cast<E*>(dst.a[i])[dest] = v[i];
    dst.key[dest] = key;
    dst.id[dest] = id;
}

constexpr int kPermPerThread = 4;

// The step's sort without moving the particle data: perm[slot] = the index
// of the particle that goes there (slots as k_scatter assigns them); the tile
// kernel then reads each particle through perm and writes it in sorted order
// into the other buffer, so the data moves once a step instead of twice.
__global__ void __launch_bounds__(kSortBlock) k_scatter_perm(const int* __restrict__ bin, int64_t np,
                                                             const int* offsets, int* count, int64_t C, int* perm,
                                                             unsigned* err) {
    // kPermPerThread particles a thread (a block's consecutive particles in
    // kPermPerThread coalesced rows): their slot atomics are in flight at once
    constexpr int U = kPermPerThread;
    const int64_t p0 = (int64_t)blockIdx.x * (U * kSortBlock) + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int k[U], base[U], old[U];
    unsigned mask[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t p = p0 + u * kSortBlock;
        k[u] = p < np ? bin[p] : -1;
        if (k[u] < 0 || k[u] >= C) k[u] = -1;
        // the bin's first slot does not depend on the atomic: loaded before it
        base[u] = k[u] >= 0 ? offsets[k[u]] : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        mask[u] = run_mask(k[u]);
        const int leader = __ffs(mask[u]) - 1;
        old[u] = 0;
        if (lane == leader && k[u] >= 0) old[u] = atomicSub(count + k[u], __popc(mask[u]));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int leader = __ffs(mask[u]) - 1;
        old[u] = __shfl_sync(0xffffffffu, old[u], leader);
        if (k[u] < 0) continue;
        const int dest = base[u] + (old[u] - __popc(mask[u])) + __popc(mask[u] & lanemask_lt());
        // checked in every build: a histogram that does not match the keys
        // (a step stopped part-way) must not send a particle outside the arrays
        if (!(dest >= 0 && dest < np)) {
            check_failed(err, 9, dest);
            continue;
        }
        perm[dest] = int(p0 + u * kSortBlock);
    }
}

// SplitMix64 output function (Steele, Lea & Flood 2014): a bijective 64-bit mixer.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Bins of pic_sort_particles: shift > 0, the cell key's run of 2^shift
// consecutive tile-major cells; shift < 0, a pseudo-random bin in [0, nb)
// from the particle id, the seed and the call counter.
__global__ void __launch_bounds__(kSortBlock) k_bin_keys(const int* __restrict__ key, const int* __restrict__ id,
                                                         int64_t np, int shift, uint64_t seed, uint64_t ctr,
                                                         int64_t nb, int* bin) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    if (shift > 0) {
        bin[p] = key[p] >> shift;
    } else {
        const uint64_t h = splitmix64(seed ^ splitmix64(uint64_t(uint32_t(id[p])) | (ctr << 32)));
        bin[p] = int(((h >> 32) * uint64_t(nb)) >> 32);
    }
}

size_t scan_status_words(int64_t C) { return size_t((C + kScanChunk - 1) / kScanChunk) + 1; }

// Bins of the sort: one per cell, plus one for removed particles when z is
// open; with pic_sort_particles' coarse bins one per run of 2^sort_shift
// cells, with its random bins one per cell.
static int64_t nbins(const pic_ctx* c) {
    if (c->sort_shift > 0) return ((c->g.C - 1) >> c->sort_shift) + 1;
    return c->g.C + (c->g.zopen ? 1 : 0);
}
static const int* bins(const pic_ctx* c) { return c->sort_shift == 0 ? c->P[c->cur].key : c->sortbin; }

cudaError_t launch_bin_keys(pic_ctx* c) {
    if (c->np == 0) return cudaSuccess;
    const unsigned nb = unsigned((c->np + kSortBlock - 1) / kSortBlock);
    k_bin_keys<<<nb, kSortBlock, 0, c->stream>>>(c->P[c->cur].key, c->P[c->cur].id, c->np, c->sort_shift, c->seed,
                                                 uint64_t(c->reorders), nbins(c), c->sortbin);
    return cudaGetLastError();
}

cudaError_t launch_hist(pic_ctx* c) {
    if (c->np == 0) return cudaSuccess;
    const unsigned nb = unsigned((c->np + kSortBlock - 1) / kSortBlock);
    k_hist<<<nb, kSortBlock, 0, c->stream>>>(bins(c), c->np, c->count, nbins(c), c->err);
    return cudaGetLastError();
}

cudaError_t launch_scan(pic_ctx* c) {
    cudaError_t e =
        cudaMemsetAsync(c->scan_status, 0, (size_t(c->scan_chunks) + 1) * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
    k_scan<<<unsigned(c->scan_chunks), kSortBlock, 0, c->stream>>>(c->count, c->offsets, nbins(c), c->scan_status,
                                                                  c->scan_chunks, c->err);
    return cudaGetLastError();
}

cudaError_t launch_scatter_perm(pic_ctx* c) {
    if (c->np == 0) return cudaSuccess;
    const unsigned nb = unsigned((c->np + kPermPerThread * kSortBlock - 1) / (kPermPerThread * kSortBlock));
    k_scatter_perm<<<nb, kSortBlock, 0, c->stream>>>(bins(c), c->np, c->offsets, c->count, nbins(c), c->perm,
                                                      c->err);
    return cudaGetLastError();
}

cudaError_t launch_scatter(pic_ctx* c) {
    if (c->np == 0) return cudaSuccess;
    const unsigned nb = unsigned((c->np + kSortBlock - 1) / kSortBlock);
    if (c->prec == PIC_FP64)
        k_scatter<double><<<nb, kSortBlock, 0, c->stream>>>(c->P[c->cur], c->P[1 - c->cur], bins(c), c->np,
                                                            c->offsets, c->count, nbins(c), c->err);
    else
        k_scatter<float><<<nb, kSortBlock, 0, c->stream>>>(c->P[c->cur], c->P[1 - c->cur], bins(c), c->np,
                                                           c->offsets, c->count, nbins(c), c->err);
    return cudaGetLastError();
}

}  // namespace pic
