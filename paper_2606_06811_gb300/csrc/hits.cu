// Seed-hit enumeration by CSR lookup (Section 2 and Section 7 seeds; the
// "position table" of Section 5). For every query position q the spaced key
// of Qs[q..q+span) is probed as is and, with transition tolerance, with each
// care position flipped to its transition partner (x ^ 2): 1 + weight probes.
// The probe keys are pairwise distinct, so a target position matches at most
// one of them and no hit is produced twice.
//
// Two passes over the same query range: count (hits per q), then an exclusive
// scan of the counts, then write (hits of q at starts[q] .. starts[q+1]). The
// write pass emits hits in increasing q, which is the order the per-diagonal
// walk needs once a stable sort groups them by diagonal.
#include "sfe_internal.cuh"

namespace sfe {

namespace {

__device__ __forceinline__ uint32_t spaced_key(const uint32_t *__restrict__ S, long long p,
                                               const SeedPattern &pat) {
    uint64_t v = (uint64_t)win16(S, p) | ((uint64_t)win16(S, p + 16) << 32);
    uint32_t k = 0;
    for (int i = 0; i < pat.weight; i++) k = (k << 2) | (uint32_t)((v >> (2 * pat.care[i])) & 3u);
    return k;
}

constexpr int MAX_PROBES = MAX_WEIGHT + 1;

// Bucket bounds of every probe of query position q, loaded together so the
// independent CSR reads overlap. Probe 0 is the exact key, probe i > 0 flips
// care position i - 1 to its transition partner.
__device__ __forceinline__ int probe_bounds(const uint32_t *__restrict__ Qs, long long q,
                                            const HitParams &hp, const uint32_t *__restrict__ off,
                                            uint32_t (&a)[MAX_PROBES], uint32_t (&b)[MAX_PROBES]) {
    const uint32_t k = spaced_key(Qs, q, hp.pat);
    const int nprobe = hp.transition ? hp.pat.weight + 1 : 1;
#pragma unroll
    for (int i = 0; i < MAX_PROBES; i++) {
        const uint32_t pk = i == 0 ? k : k ^ (2u << (2 * (i - 1)));
        a[i] = i < nprobe ? __ldg(off + pk) : 0u;
        b[i] = i < nprobe ? __ldg(off + pk + 1) : 0u;
    }
    return nprobe;
}

// Hits of every key's probe set (the key and, with transitions, its weight
// transition variants), from the CSR offsets: the count pass then reads one
// word per query position instead of 1 + weight bucket bounds.
__global__ void neighbor_count_kernel(const uint32_t *__restrict__ off, int weight,
                                      int transition, uint32_t *__restrict__ ncount) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= (1LL << (2 * weight))) return;
    uint32_t c = __ldg(off + k + 1) - __ldg(off + k);
    if (transition)
        for (int i = 0; i < weight; i++) {
            const long long p = k ^ (2LL << (2 * i));
            c += __ldg(off + p + 1) - __ldg(off + p);
        }
    ncount[k] = c;
}

__global__ void __launch_bounds__(BLOCK) hit_count_table_kernel(const uint32_t *__restrict__ Qs,
                                                                HitParams hp,
                                                                const uint32_t *__restrict__ ncount,
                                                                long long q0, long long q1,
                                                                uint32_t *__restrict__ counts) {
    long long q = q0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= q1) return;
    counts[q - q0] = __ldg(ncount + spaced_key(Qs, q, hp.pat));
}

__global__ void __launch_bounds__(BLOCK) hit_count_kernel(const uint32_t *__restrict__ Qs,
                                                          HitParams hp,
                                                          const uint32_t *__restrict__ off,
                                                          long long q0, long long q1,
                                                          uint32_t *__restrict__ counts) {
    long long q = q0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= q1) return;
    uint32_t a[MAX_PROBES], b[MAX_PROBES];
    probe_bounds(Qs, q, hp, off, a, b);
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < MAX_PROBES; i++) c += b[i] - a[i];
    counts[q - q0] = c;
}

// Sparse index (a heavy seed on a target that fills few of its 4^weight
// keys): the CSR is over each key's top bits, about one entry per bucket, so
// its offsets stay in L2; entry j keeps the rest of its key in low[j]. A
// probe reads its bucket's bounds and counts (or writes) the entries whose
// low bits are its own. Entries of one key are contiguous and in position
// order (the index is sorted by key, then position).
__global__ void __launch_bounds__(BLOCK) hit_count_sparse_kernel(
    const uint32_t *__restrict__ Qs, HitParams hp, const uint32_t *__restrict__ off,
    long long q0, long long q1, uint32_t *__restrict__ counts) {
    long long q = q0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= q1) return;
    const uint32_t k = spaced_key(Qs, q, hp.pat);
    const int nprobe = hp.transition ? hp.pat.weight + 1 : 1;
    const uint32_t lmask = (1u << hp.shift) - 1u;
    uint32_t a[MAX_PROBES], b[MAX_PROBES];
#pragma unroll
    for (int i = 0; i < MAX_PROBES; i++) {
        const uint32_t pk = i == 0 ? k : k ^ (2u << (2 * (i - 1)));
        a[i] = i < nprobe ? __ldg(off + (pk >> hp.shift)) : 0u;
        b[i] = i < nprobe ? __ldg(off + (pk >> hp.shift) + 1) : 0u;
    }
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < MAX_PROBES; i++) {
        const uint32_t lo = (i == 0 ? k : k ^ (2u << (2 * (i - 1)))) & lmask;
        for (uint32_t j = a[i]; j < b[i]; j++) c += __ldg(hp.low + j) == lo;
    }
    counts[q - q0] = c;
}

__global__ void __launch_bounds__(BLOCK) hit_write_sparse_kernel(
    const uint32_t *__restrict__ Qs, HitParams hp, const uint32_t *__restrict__ off,
    const uint32_t *__restrict__ pos, long long q0, long long q1,
    const unsigned long long *__restrict__ starts, unsigned long long base,
    uint64_t *__restrict__ hits) {
    long long q = q0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= q1) return;
    const uint32_t k = spaced_key(Qs, q, hp.pat);
    const int nprobe = hp.transition ? hp.pat.weight + 1 : 1;
    const uint32_t lmask = (1u << hp.shift) - 1u;
    uint32_t a[MAX_PROBES], b[MAX_PROBES];
#pragma unroll
    for (int i = 0; i < MAX_PROBES; i++) {
        const uint32_t pk = i == 0 ? k : k ^ (2u << (2 * (i - 1)));
        a[i] = i < nprobe ? __ldg(off + (pk >> hp.shift)) : 0u;
        b[i] = i < nprobe ? __ldg(off + (pk >> hp.shift) + 1) : 0u;
    }
    unsigned long long o = starts[q - q0] - base;
    const long long dq = hp.qoff - q;  // D = t + dq
#pragma unroll
    for (int i = 0; i < MAX_PROBES; i++) {
        const uint32_t lo = (i == 0 ? k : k ^ (2u << (2 * (i - 1)))) & lmask;
        for (uint32_t j = a[i]; j < b[i]; j++) {
            if (__ldg(hp.low + j) != lo) continue;
            const uint32_t t = __ldg(pos + j);
            __stcs(reinterpret_cast<unsigned long long *>(hits) + o++,
                   (unsigned long long)make_hit((uint32_t)(t + dq), t));
        }
    }
}

// Hits go out with evict-first stores: the stream of hit records must not push
// the CSR table out of L2. Each thread writes the hits of its query position.
__global__ void __launch_bounds__(BLOCK) hit_write_kernel(
    const uint32_t *__restrict__ Qs, HitParams hp, const uint32_t *__restrict__ off,
    const uint32_t *__restrict__ pos, long long q0, long long q1,
    const unsigned long long *__restrict__ starts, unsigned long long base,
    uint64_t *__restrict__ hits) {
    long long q = q0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= q1) return;
    uint32_t a[MAX_PROBES], b[MAX_PROBES];
    probe_bounds(Qs, q, hp, off, a, b);
    unsigned long long o = starts[q - q0] - base;
    const long long dq = hp.qoff - q;  // D = t + dq
#pragma unroll
    for (int i = 0; i < MAX_PROBES; i++) {  // unused probes have empty buckets
        for (uint32_t j = a[i]; j < b[i]; j++) {
            const uint32_t t = __ldg(pos + j);
            __stcs(reinterpret_cast<unsigned long long *>(hits) + o++,
                   (unsigned long long)make_hit((uint32_t)(t + dq), t));
        }
    }
}

// The same output, for query ranges with many hits per position (repeat
// families, long homologous blocks): one warp writes the hits of its 32 query
// positions together. The warp's output range is contiguous and in q order
// (lane order, then probe order, then bucket order), so output slot k of the
// warp is found by two small searches in shared memory (the lane, then the
// probe), and the position reads and hit writes of consecutive slots are
// consecutive. The set-up costs shared memory and registers, so positions
// with few hits are faster with the kernel above.
constexpr int HW_WARPS = BLOCK / 32;

__global__ void __launch_bounds__(BLOCK) hit_write_warp_kernel(
    const uint32_t *__restrict__ Qs, HitParams hp, const uint32_t *__restrict__ off,
    const uint32_t *__restrict__ pos, long long q0, long long q1,
    const unsigned long long *__restrict__ starts, unsigned long long base,
    uint64_t *__restrict__ hits) {
    __shared__ uint32_t s_a[HW_WARPS][32][MAX_PROBES];      // bucket starts
    __shared__ uint32_t s_p[HW_WARPS][32][MAX_PROBES + 1];  // lane's exclusive prefix over probes
    __shared__ uint32_t s_o[HW_WARPS][33];                  // warp's exclusive prefix over lanes
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long qw = q0 + (blockIdx.x * (long long)blockDim.x) + w * 32;  // lane 0's q
    if (qw >= q1) return;
    const long long q = qw + lane;
    uint32_t a[MAX_PROBES], b[MAX_PROBES];
    if (q < q1) {
        probe_bounds(Qs, q, hp, off, a, b);
    } else {
#pragma unroll
        for (int i = 0; i < MAX_PROBES; i++) a[i] = b[i] = 0u;
    }
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < MAX_PROBES; i++) {
        s_a[w][lane][i] = a[i];
        s_p[w][lane][i] = c;
        c += b[i] - a[i];
    }
    s_p[w][lane][MAX_PROBES] = c;
    uint32_t incl = c;  // a warp's hits lie in one query tile (checked: < 2^32)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    s_o[w][lane] = incl - c;
    if (lane == 31) s_o[w][32] = incl;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const unsigned long long wbase = starts[qw - q0] - base;
    __syncwarp();
    for (uint32_t k = lane; k < total; k += 32) {
        int L = 0;  // last lane whose range starts at or before k
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
            if (s_o[w][L + step] <= k) L += step;
        const uint32_t r = k - s_o[w][L];
        int i = 0;  // last probe whose range starts at or before r
#pragma unroll
        for (int step = 8; step > 0; step >>= 1)
            if (i + step < MAX_PROBES && s_p[w][L][i + step] <= r) i += step;
        const uint32_t t = __ldg(pos + s_a[w][L][i] + (r - s_p[w][L][i]));
        const long long dq = hp.qoff - (qw + L);  // D = t + dq
        __stcs(reinterpret_cast<unsigned long long *>(hits) + wbase + k,
               (unsigned long long)make_hit((uint32_t)(t + dq), t));
    }
}

// Merged probe-set lists: for every key, the positions of all the buckets its
// probe set reads, back to back (probe order, then bucket order), so writing
// the hits of a query position copies one contiguous range.
__global__ void merged_fill_kernel(const uint32_t *__restrict__ off,
                                   const uint32_t *__restrict__ pos, int weight, int transition,
                                   const uint32_t *__restrict__ off2, uint32_t *__restrict__ pos2) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= (1LL << (2 * weight))) return;
    uint32_t o = off2[k];
    const int nprobe = transition ? weight + 1 : 1;
    for (int i = 0; i < nprobe; i++) {
        const long long p = i == 0 ? k : (k ^ (2LL << (2 * (i - 1))));
        for (uint32_t j = __ldg(off + p); j < __ldg(off + p + 1); j++) pos2[o++] = __ldg(pos + j);
    }
}

// Writer over merged lists, one warp per 32 query positions: one range per
// lane, so an output slot needs only the search for its lane, and the reads
// and writes of consecutive slots are consecutive.
__global__ void __launch_bounds__(BLOCK) hit_write_merged_warp_kernel(
    const uint32_t *__restrict__ Qs, HitParams hp, const uint32_t *__restrict__ off2,
    const uint32_t *__restrict__ pos2, long long q0, long long q1,
    const unsigned long long *__restrict__ starts, unsigned long long base,
    uint64_t *__restrict__ hits) {
    __shared__ uint32_t s_a[HW_WARPS][32];
    __shared__ uint32_t s_o[HW_WARPS][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long qw = q0 + (blockIdx.x * (long long)blockDim.x) + w * 32;
    if (qw >= q1) return;
    const long long q = qw + lane;
    uint32_t a = 0, c = 0;
    if (q < q1) {
        const uint32_t k = spaced_key(Qs, q, hp.pat);
        a = __ldg(off2 + k);
        c = __ldg(off2 + k + 1) - a;
    }
    uint32_t incl = c;  // a warp's hits lie in one query tile (checked: < 2^32)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    s_a[w][lane] = a;
    s_o[w][lane] = incl - c;
    if (lane == 31) s_o[w][32] = incl;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const unsigned long long wbase = starts[qw - q0] - base;
    __syncwarp();
    for (uint32_t k = lane; k < total; k += 32) {
        int L = 0;  // last lane whose range starts at or before k
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
            if (s_o[w][L + step] <= k) L += step;
        const uint32_t t = __ldg(pos2 + s_a[w][L] + (k - s_o[w][L]));
        const long long dq = hp.qoff - (qw + L);
        __stcs(reinterpret_cast<unsigned long long *>(hits) + wbase + k,
               (unsigned long long)make_hit((uint32_t)(t + dq), t));
    }
}

inline unsigned grid_for(long long n) { return (unsigned)((n + BLOCK - 1) / BLOCK); }

}  // namespace

cudaError_t launch_neighbor_counts(const uint32_t *offsets, const SeedPattern &pat,
                                   int transition, uint32_t *ncount, cudaStream_t st) {
    g_launches++;
    neighbor_count_kernel<<<grid_for(1LL << (2 * pat.weight)), BLOCK, 0, st>>>(
        offsets, pat.weight, transition, ncount);
    return cudaGetLastError();
}

cudaError_t launch_hit_count(const uint32_t *Qs, HitParams hp, const uint32_t *offsets,
                             const uint32_t *ncount, long long q0, long long q1, uint32_t *counts,
                             cudaStream_t st) {
    if (q1 <= q0) return cudaSuccess;
    g_launches++;
    if (hp.low)
        hit_count_sparse_kernel<<<grid_for(q1 - q0), BLOCK, 0, st>>>(Qs, hp, offsets, q0, q1,
                                                                     counts);
    else if (ncount)
        hit_count_table_kernel<<<grid_for(q1 - q0), BLOCK, 0, st>>>(Qs, hp, ncount, q0, q1,
                                                                    counts);
    else
        hit_count_kernel<<<grid_for(q1 - q0), BLOCK, 0, st>>>(Qs, hp, offsets, q0, q1, counts);
    return cudaGetLastError();
}

cudaError_t launch_merged_fill(const uint32_t *offsets, const uint32_t *positions,
                               const SeedPattern &pat, int transition, const uint32_t *off2,
                               uint32_t *pos2, cudaStream_t st) {
    g_launches++;
    merged_fill_kernel<<<grid_for(1LL << (2 * pat.weight)), BLOCK, 0, st>>>(
        offsets, positions, pat.weight, transition, off2, pos2);
    return cudaGetLastError();
}

cudaError_t launch_hit_write(const uint32_t *Qs, HitParams hp, const uint32_t *offsets,
                             const uint32_t *positions, const uint32_t *off2,
                             const uint32_t *pos2, long long q0, long long q1,
                             const unsigned long long *starts, unsigned long long base,
                             unsigned long long nhits, uint64_t *hits, cudaStream_t st) {
    if (q1 <= q0) return cudaSuccess;
    g_launches++;
    if (hp.low) {
        hit_write_sparse_kernel<<<grid_for(q1 - q0), BLOCK, 0, st>>>(Qs, hp, offsets, positions,
                                                                     q0, q1, starts, base, hits);
        return cudaGetLastError();
    }
    if (off2) {
        // with one range per position the per-warp writer wins even at a few
        // hits per position (10 Mb pair: 0.95 against 2.05 ms per step)
        hit_write_merged_warp_kernel<<<grid_for(q1 - q0), BLOCK, 0, st>>>(Qs, hp, off2, pos2, q0,
                                                                          q1, starts, base, hits);
        return cudaGetLastError();
    }
    // measured: ~10 hits per position (the 10 Mb pair) is faster per thread,
    // ~95 (the 100 Mb pair's repeats) per warp
    if (nhits >= 32ull * (unsigned long long)(q1 - q0))
        hit_write_warp_kernel<<<grid_for(q1 - q0), BLOCK, 0, st>>>(Qs, hp, offsets, positions,
                                                                   q0, q1, starts, base, hits);
    else
        hit_write_kernel<<<grid_for(q1 - q0), BLOCK, 0, st>>>(Qs, hp, offsets, positions, q0, q1,
                                                              starts, base, hits);
    return cudaGetLastError();
}

}  // namespace sfe
