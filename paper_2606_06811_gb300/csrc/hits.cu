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

__global__ void __launch_bounds__(BLOCK) hit_count_kernel(const uint32_t *__restrict__ Qs,
                                                          HitParams hp,
                                                          const uint32_t *__restrict__ off,
                                                          long long q0, long long q1,
                                                          uint32_t *__restrict__ counts) {
    long long q = q0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= q1) return;
    uint32_t k = spaced_key(Qs, q, hp.pat);
    uint32_t c = __ldg(off + k + 1) - __ldg(off + k);
    if (hp.transition) {
        for (int i = 0; i < hp.pat.weight; i++) {
            uint32_t pk = k ^ (2u << (2 * i));
            c += __ldg(off + pk + 1) - __ldg(off + pk);
        }
    }
    counts[q - q0] = c;
}

__global__ void __launch_bounds__(BLOCK) hit_write_kernel(
    const uint32_t *__restrict__ Qs, HitParams hp, const uint32_t *__restrict__ off,
    const uint32_t *__restrict__ pos, long long q0, long long q1,
    const unsigned long long *__restrict__ starts, unsigned long long base,
    uint64_t *__restrict__ hits) {
    long long q = q0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= q1) return;
    uint32_t k = spaced_key(Qs, q, hp.pat);
    unsigned long long o = starts[q - q0] - base;
    const long long dq = hp.qoff - q;  // D = t + dq
    int nprobe = hp.transition ? hp.pat.weight + 1 : 1;
    for (int i = 0; i < nprobe; i++) {
        uint32_t pk = i == 0 ? k : k ^ (2u << (2 * (i - 1)));
        uint32_t a = __ldg(off + pk), b = __ldg(off + pk + 1);
        for (uint32_t j = a; j < b; j++) {
            uint32_t t = __ldg(pos + j);
            hits[o++] = make_hit((uint32_t)(t + dq), t);
        }
    }
}

inline unsigned grid_for(long long n) { return (unsigned)((n + BLOCK - 1) / BLOCK); }

}  // namespace

cudaError_t launch_hit_count(const uint32_t *Qs, HitParams hp, const uint32_t *offsets,
                             long long q0, long long q1, uint32_t *counts, cudaStream_t st) {
    if (q1 <= q0) return cudaSuccess;
    hit_count_kernel<<<grid_for(q1 - q0), BLOCK, 0, st>>>(Qs, hp, offsets, q0, q1, counts);
    return cudaGetLastError();
}

cudaError_t launch_hit_write(const uint32_t *Qs, HitParams hp, const uint32_t *offsets,
                             const uint32_t *positions, long long q0, long long q1,
                             const unsigned long long *starts, unsigned long long base,
                             uint64_t *hits, cudaStream_t st) {
    if (q1 <= q0) return cudaSuccess;
    hit_write_kernel<<<grid_for(q1 - q0), BLOCK, 0, st>>>(Qs, hp, offsets, positions, q0, q1,
                                                          starts, base, hits);
    return cudaGetLastError();
}

}  // namespace sfe
