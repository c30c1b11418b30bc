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

// Hits go out with evict-first stores: the stream of hit records must not push
// the CSR table out of L2.
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

inline unsigned grid_for(long long n) { return (unsigned)((n + BLOCK - 1) / BLOCK); }

}  // namespace

cudaError_t launch_hit_count(const uint32_t *Qs, HitParams hp, const uint32_t *offsets,
                             long long q0, long long q1, uint32_t *counts, cudaStream_t st) {
    if (q1 <= q0) return cudaSuccess;
    g_launches++;
    hit_count_kernel<<<grid_for(q1 - q0), BLOCK, 0, st>>>(Qs, hp, offsets, q0, q1, counts);
    return cudaGetLastError();
}

cudaError_t launch_hit_write(const uint32_t *Qs, HitParams hp, const uint32_t *offsets,
                             const uint32_t *positions, long long q0, long long q1,
                             const unsigned long long *starts, unsigned long long base,
                             uint64_t *hits, cudaStream_t st) {
    if (q1 <= q0) return cudaSuccess;
    g_launches++;
    hit_write_kernel<<<grid_for(q1 - q0), BLOCK, 0, st>>>(Qs, hp, offsets, positions, q0, q1,
                                                          starts, base, hits);
    return cudaGetLastError();
}

}  // namespace sfe
