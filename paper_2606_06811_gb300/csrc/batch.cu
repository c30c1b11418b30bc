// Seeding and HSP ordering for a batch of target/query pairs.
//
// Every pair has its own seeding index, so no hit ever joins two pairs. A pair
// with n seed positions gets 2^b buckets, b = ceil(log2 n) clamped to
// [4, 2 * weight], addressed by the top b bits of the seed key; the buckets of
// all pairs sit back to back in one CSR table. Entries keep their full key, so
// a probe scans its bucket (on average under one entry) and keeps the entries
// whose key is equal. The table is filled by a counting sort (counts, one
// exclusive scan over all pairs' buckets, atomic placement): the order of the
// entries inside a bucket is not fixed, and it need not be, because hits of
// one query position lie on different diagonals and the diagonal grouping that
// follows only relies on query order within a diagonal.
//
// Hit words: pair << (dbits + 1) | strand << dbits | local diagonal in the
// high half, local t in the low half, written in query order per (pair,
// strand) so a stable sort on the high half groups each diagonal in t order.
#include "sfe_internal.cuh"

namespace sfe {

namespace {

constexpr int MAX_PROBES = MAX_WEIGHT + 1;

__device__ __forceinline__ uint32_t spaced_key(const uint32_t *__restrict__ S, long long p,
                                               const SeedPattern &pat) {
    uint64_t v = (uint64_t)win16(S, p) | ((uint64_t)win16(S, p + 16) << 32);
    uint32_t k = 0;
    for (int i = 0; i < pat.weight; i++) k = (k << 2) | (uint32_t)((v >> (2 * pat.care[i])) & 3u);
    return k;
}

// One block per pair: bucket sizes of its index.
__global__ void __launch_bounds__(BLOCK) bidx_count(const uint32_t *__restrict__ T,
                                                    const PairInfo *__restrict__ pairs,
                                                    SeedPattern pat, uint32_t *__restrict__ cnt) {
    const PairInfo P = pairs[blockIdx.x];
    const long long npos = (long long)P.tlen - pat.span + 1;
    const int kbits = 2 * pat.weight;
    for (long long i = threadIdx.x; i < npos; i += BLOCK) {
        const uint32_t k = spaced_key(T, P.toff + i, pat);
        atomicAdd(cnt + P.boff + (k >> (kbits - P.bbits)), 1u);
    }
}

// One block per pair: entries (key << 32 | local position) in their buckets.
__global__ void __launch_bounds__(BLOCK) bidx_fill(const uint32_t *__restrict__ T,
                                                   const PairInfo *__restrict__ pairs,
                                                   SeedPattern pat,
                                                   const uint32_t *__restrict__ off,
                                                   uint32_t *__restrict__ cursor,
                                                   uint64_t *__restrict__ entries) {
    const PairInfo P = pairs[blockIdx.x];
    const long long npos = (long long)P.tlen - pat.span + 1;
    const int kbits = 2 * pat.weight;
    for (long long i = threadIdx.x; i < npos; i += BLOCK) {
        const uint32_t k = spaced_key(T, P.toff + i, pat);
        const long long b = P.boff + (k >> (kbits - P.bbits));
        const uint32_t slot = off[b] + atomicAdd(cursor + b, 1u);
        entries[slot] = ((uint64_t)k << 32) | (uint32_t)i;
    }
}

// Hits of query position q (pair P, strand s) against P's index: counted, or
// written from `o` on when `out` is given.
template <bool WRITE>
__device__ __forceinline__ uint32_t bhits_at(const uint32_t *__restrict__ Qs, long long qg,
                                             long long q, const PairInfo &P, int pair, int s,
                                             const SeedPattern &pat, int transition, int dbits,
                                             const uint32_t *__restrict__ off,
                                             const uint64_t *__restrict__ entries,
                                             uint64_t *__restrict__ out, unsigned long long o) {
    const uint32_t k = spaced_key(Qs, qg, pat);
    const int kbits = 2 * pat.weight;
    const int nprobe = transition ? pat.weight + 1 : 1;
    const uint32_t hi_base = ((uint32_t)pair << (dbits + 1)) | ((uint32_t)s << dbits);
    const long long dq = (long long)P.qlen - pat.span - q;  // D = t + dq
    uint32_t c = 0;
    for (int i = 0; i < nprobe; i++) {
        const uint32_t pk = i == 0 ? k : k ^ (2u << (2 * (i - 1)));
        const long long b = P.boff + (pk >> (kbits - P.bbits));
        const uint32_t a = __ldg(off + b), e = __ldg(off + b + 1);
        for (uint32_t j = a; j < e; j++) {
            const uint64_t ent = __ldg(entries + j);
            if ((uint32_t)(ent >> 32) != pk) continue;
            if (WRITE) {
                const uint32_t t = (uint32_t)ent;
                out[o + c] = ((uint64_t)(hi_base | (uint32_t)(t + dq)) << 32) | t;
            }
            c++;
        }
    }
    return c;
}

// Grid (pair, strand): counts[s * qtotal + qoff + q] for every query position.
__global__ void __launch_bounds__(BLOCK) bhits_count(const uint32_t *__restrict__ Q,
                                                     const uint32_t *__restrict__ Qrc,
                                                     const PairInfo *__restrict__ pairs,
                                                     int strands, SeedPattern pat, int transition,
                                                     int dbits,
                                                     long long qtotal,
                                                     const uint32_t *__restrict__ off,
                                                     const uint64_t *__restrict__ entries,
                                                     uint32_t *__restrict__ counts) {
    const int pair = blockIdx.x, s = blockIdx.y;
    if (!((strands >> s) & 1)) return;
    const PairInfo P = pairs[pair];
    const uint32_t *Qs = s ? Qrc : Q;
    const long long qb = s ? P.qoff_rc : P.qoff;
    const long long nq = (long long)P.qlen - pat.span + 1;
    if ((long long)P.tlen < pat.span) return;
    for (long long q = threadIdx.x; q < nq; q += BLOCK)
        counts[s * qtotal + P.qoff + q] = bhits_at<false>(Qs, qb + q, q, P, pair, s, pat,
                                                          transition, dbits, off, entries,
                                                          nullptr, 0);
}

__global__ void __launch_bounds__(BLOCK) bhits_write(const uint32_t *__restrict__ Q,
                                                     const uint32_t *__restrict__ Qrc,
                                                     const PairInfo *__restrict__ pairs,
                                                     int strands, SeedPattern pat, int transition,
                                                     int dbits,
                                                     long long qtotal,
                                                     const uint32_t *__restrict__ off,
                                                     const uint64_t *__restrict__ entries,
                                                     const unsigned long long *__restrict__ starts,
                                                     uint64_t *__restrict__ hits) {
    const int pair = blockIdx.x, s = blockIdx.y;
    if (!((strands >> s) & 1)) return;
    const PairInfo P = pairs[pair];
    const uint32_t *Qs = s ? Qrc : Q;
    const long long qb = s ? P.qoff_rc : P.qoff;
    const long long nq = (long long)P.qlen - pat.span + 1;
    if ((long long)P.tlen < pat.span) return;
    for (long long q = threadIdx.x; q < nq; q += BLOCK)
        bhits_at<true>(Qs, qb + q, q, P, pair, s, pat, transition, dbits, off, entries, hits,
                       starts[s * qtotal + P.qoff + q]);
}

// ---------------------------------------------------------------- HSP order

__global__ void bhsp_keys(const BatchHsp *__restrict__ h, long long n, int lbits,
                          uint64_t *__restrict__ keys, unsigned *__restrict__ idx) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const BatchHsp x = h[i];
    keys[i] = ((uint64_t)(uint32_t)x.pair << (2 * lbits + 1)) |
              ((uint64_t)(uint32_t)x.strand << (2 * lbits)) |
              ((uint64_t)(uint32_t)x.tpos << lbits) | (uint64_t)(uint32_t)x.qpos;
    idx[i] = (unsigned)i;
}

__global__ void bhsp_gather(const BatchHsp *__restrict__ h, const unsigned *__restrict__ idx,
                            long long n, BatchHsp *__restrict__ out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = h[idx[i]];
}

__device__ __forceinline__ bool bhsp_less(const BatchHsp &a, const BatchHsp &b) {
    if (a.len != b.len) return a.len < b.len;
    return a.score < b.score;
}

// Runs of equal (pair, strand, tpos, qpos) ordered by (len, score).
__global__ void bhsp_fix_runs(BatchHsp *__restrict__ h, const uint64_t *__restrict__ keys,
                              long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i > 0 && keys[i - 1] == keys[i]) return;
    long long j = i + 1;
    while (j < n && keys[j] == keys[i]) j++;
    for (long long a = i + 1; a < j; a++) {
        BatchHsp x = h[a];
        long long b = a - 1;
        while (b >= i && bhsp_less(x, h[b])) {
            h[b + 1] = h[b];
            b--;
        }
        h[b + 1] = x;
    }
}

inline unsigned grid_for(long long n) { return (unsigned)((n + BLOCK - 1) / BLOCK); }

}  // namespace

cudaError_t launch_batch_index(const uint32_t *T, const PairInfo *pairs, int npairs,
                               SeedPattern pat, uint32_t *cnt, long long nbuckets, uint32_t *off,
                               uint64_t *entries, void *tmp, cudaStream_t st) {
    cudaMemsetAsync(cnt, 0, (size_t)nbuckets * 4, st);
    g_launches++;
    bidx_count<<<npairs, BLOCK, 0, st>>>(T, pairs, pat, cnt);
    cudaError_t e = scan_u32_to_u32(cnt, off, nbuckets, tmp, st);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(cnt, 0, (size_t)nbuckets * 4, st);  // reused as placement cursors
    g_launches++;
    bidx_fill<<<npairs, BLOCK, 0, st>>>(T, pairs, pat, off, cnt, entries);
    return cudaGetLastError();
}

cudaError_t launch_batch_hit_count(const uint32_t *Q, const uint32_t *Qrc, const PairInfo *pairs,
                                   int npairs, int strands_mask, SeedPattern pat, int transition,
                                   int dbits, long long qtotal, const uint32_t *off,
                                   const uint64_t *entries, uint32_t *counts, cudaStream_t st) {
    cudaMemsetAsync(counts, 0, (size_t)(2 * qtotal) * 4, st);
    dim3 grid(npairs, 2);
    g_launches++;
    bhits_count<<<grid, BLOCK, 0, st>>>(Q, Qrc, pairs, strands_mask, pat, transition, dbits,
                                        qtotal, off, entries, counts);
    return cudaGetLastError();
}

cudaError_t launch_batch_hit_write(const uint32_t *Q, const uint32_t *Qrc, const PairInfo *pairs,
                                   int npairs, int strands_mask, SeedPattern pat, int transition,
                                   int dbits, long long qtotal, const uint32_t *off,
                                   const uint64_t *entries, const unsigned long long *starts,
                                   uint64_t *hits, cudaStream_t st) {
    dim3 grid(npairs, 2);
    g_launches++;
    bhits_write<<<grid, BLOCK, 0, st>>>(Q, Qrc, pairs, strands_mask, pat, transition, dbits,
                                        qtotal, off, entries, starts, hits);
    return cudaGetLastError();
}

size_t batch_hsp_sort_temp_bytes(long long n) {
    n = n > 0 ? n : 1;
    return (size_t)n * (8 + 8 + 4 + 4 + sizeof(BatchHsp)) + radix_sort_temp_bytes(n) + 1536;
}

cudaError_t batch_hsp_sort(BatchHsp *h, long long n, int pbits, int lbits, void *tmp,
                           uint32_t *status, cudaStream_t st) {
    if (n <= 1) return cudaSuccess;
    char *p = reinterpret_cast<char *>(tmp);
    auto take = [&](size_t bytes) {
        char *r = p;
        p += (bytes + 255) & ~(size_t)255;
        return r;
    };
    uint64_t *ka = reinterpret_cast<uint64_t *>(take((size_t)n * 8));
    uint64_t *kb = reinterpret_cast<uint64_t *>(take((size_t)n * 8));
    unsigned *va = reinterpret_cast<unsigned *>(take((size_t)n * 4));
    unsigned *vb = reinterpret_cast<unsigned *>(take((size_t)n * 4));
    BatchHsp *hb = reinterpret_cast<BatchHsp *>(take((size_t)n * sizeof(BatchHsp)));
    void *rt = take(radix_sort_temp_bytes(n));
    g_launches++;
    bhsp_keys<<<grid_for(n), BLOCK, 0, st>>>(h, n, lbits, ka, va);
    bool in_b = false;
    cudaError_t e = radix_sort(ka, kb, va, vb, n, 0, pbits + 1 + 2 * lbits, rt, &in_b, status, st);
    if (e != cudaSuccess) return e;
    uint64_t *kf = in_b ? kb : ka;
    unsigned *vf = in_b ? vb : va;
    g_launches += 2;
    bhsp_gather<<<grid_for(n), BLOCK, 0, st>>>(h, vf, n, hb);
    bhsp_fix_runs<<<grid_for(n), BLOCK, 0, st>>>(hb, kf, n);
    cudaMemcpyAsync(h, hb, (size_t)n * sizeof(BatchHsp), cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError();
}

}  // namespace sfe
