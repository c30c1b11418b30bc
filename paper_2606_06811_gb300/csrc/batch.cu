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

// Work items: fixed-size chunks of one pair's positions, numbered pair by
// pair, so the CTAs in flight at any moment touch only a few consecutive pairs
// and their index buckets stay in L2. prefix[p] = first item of pair p.
constexpr int ITEM = 1024;  // positions per work item

__device__ __forceinline__ int item_pair(const long long *__restrict__ prefix, int npairs,
                                         long long item) {
    int lo = 0, hi = npairs;  // last p with prefix[p] <= item
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (prefix[mid] <= item)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Bucket sizes of every pair's index, one work item per block.
__global__ void __launch_bounds__(BLOCK) bidx_count(const uint32_t *__restrict__ T,
                                                    const PairInfo *__restrict__ pairs,
                                                    const long long *__restrict__ tprefix,
                                                    int npairs, SeedPattern pat,
                                                    uint32_t *__restrict__ cnt) {
    const int p = item_pair(tprefix, npairs, blockIdx.x);
    const PairInfo P = pairs[p];
    const long long npos = (long long)P.tlen - pat.span + 1;
    const long long i0 = (blockIdx.x - tprefix[p]) * (long long)ITEM;
    const int kbits = 2 * pat.weight;
    for (long long i = i0 + threadIdx.x; i < min(npos, i0 + ITEM); i += BLOCK) {
        const uint32_t k = spaced_key(T, P.toff + i, pat);
        atomicAdd(cnt + P.boff + (k >> (kbits - P.bbits)), 1u);
    }
}

// Entries (key << 32 | local position) in their buckets, one work item per block.
__global__ void __launch_bounds__(BLOCK) bidx_fill(const uint32_t *__restrict__ T,
                                                   const PairInfo *__restrict__ pairs,
                                                   const long long *__restrict__ tprefix,
                                                   int npairs, SeedPattern pat,
                                                   const uint32_t *__restrict__ off,
                                                   uint32_t *__restrict__ cursor,
                                                   uint64_t *__restrict__ entries) {
    const int p = item_pair(tprefix, npairs, blockIdx.x);
    const PairInfo P = pairs[p];
    const long long npos = (long long)P.tlen - pat.span + 1;
    const long long i0 = (blockIdx.x - tprefix[p]) * (long long)ITEM;
    const int kbits = 2 * pat.weight;
    for (long long i = i0 + threadIdx.x; i < min(npos, i0 + ITEM); i += BLOCK) {
        const uint32_t k = spaced_key(T, P.toff + i, pat);
        const long long b = P.boff + (k >> (kbits - P.bbits));
        const uint32_t slot = off[b] + atomicAdd(cursor + b, 1u);
        entries[slot] = ((uint64_t)k << 32) | (uint32_t)i;
    }
}

// Hits of query position q (pair P, strand s) against P's index: counted, or
// written from `o` on when WRITE. The bucket bounds of all probes are loaded
// together so the independent reads overlap; then each bucket is scanned for
// entries whose key is the probe's.
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
    uint32_t pk[MAX_PROBES], a[MAX_PROBES], e[MAX_PROBES];
#pragma unroll
    for (int i = 0; i < MAX_PROBES; i++) {
        pk[i] = i == 0 ? k : k ^ (2u << (2 * (i - 1)));
        const long long b = P.boff + (pk[i] >> (kbits - P.bbits));
        a[i] = i < nprobe ? __ldg(off + b) : 0u;
        e[i] = i < nprobe ? __ldg(off + b + 1) : 0u;
    }
    const uint32_t hi_base = ((uint32_t)pair << (dbits + 1)) | ((uint32_t)s << dbits);
    const long long dq = (long long)P.qlen - pat.span - q;  // D = t + dq
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < MAX_PROBES; i++) {
        for (uint32_t j = a[i]; j < e[i]; j++) {
            const uint64_t ent = __ldg(entries + j);
            if ((uint32_t)(ent >> 32) != pk[i]) continue;
            if (WRITE) {
                const uint32_t t = (uint32_t)ent;
                out[o + c] = ((uint64_t)(hi_base | (uint32_t)(t + dq)) << 32) | t;
            }
            c++;
        }
    }
    return c;
}

// Work item of the query side: (pair, strand, chunk), both strands of a pair
// next to each other; qprefix[p] = first item of pair p.
__device__ __forceinline__ void query_item(const long long *__restrict__ qprefix, int npairs,
                                           long long item, int &p, int &s, long long &q0) {
    p = item_pair(qprefix, npairs, item);
    const long long local = item - qprefix[p];
    s = (int)(local & 1);
    q0 = (local >> 1) * ITEM;
}

// counts[s * qtotal + qoff + q] for every query position of every item.
__global__ void __launch_bounds__(BLOCK) bhits_count(const uint32_t *__restrict__ Q,
                                                     const uint32_t *__restrict__ Qrc,
                                                     const PairInfo *__restrict__ pairs,
                                                     const long long *__restrict__ qprefix,
                                                     int npairs, int strands, SeedPattern pat,
                                                     int transition, int dbits, long long qtotal,
                                                     const uint32_t *__restrict__ off,
                                                     const uint64_t *__restrict__ entries,
                                                     uint32_t *__restrict__ counts) {
    int pair, s;
    long long q0;
    query_item(qprefix, npairs, blockIdx.x, pair, s, q0);
    if (!((strands >> s) & 1)) return;
    const PairInfo P = pairs[pair];
    if ((long long)P.tlen < pat.span) return;
    const uint32_t *Qs = s ? Qrc : Q;
    const long long qb = s ? P.qoff_rc : P.qoff;
    const long long nq = (long long)P.qlen - pat.span + 1;
    for (long long q = q0 + threadIdx.x; q < min(nq, q0 + ITEM); q += BLOCK)
        counts[s * qtotal + P.qoff + q] = bhits_at<false>(Qs, qb + q, q, P, pair, s, pat,
                                                          transition, dbits, off, entries,
                                                          nullptr, 0);
}

__global__ void __launch_bounds__(BLOCK) bhits_write(const uint32_t *__restrict__ Q,
                                                     const uint32_t *__restrict__ Qrc,
                                                     const PairInfo *__restrict__ pairs,
                                                     const long long *__restrict__ qprefix,
                                                     int npairs, int strands, SeedPattern pat,
                                                     int transition, int dbits, long long qtotal,
                                                     const uint32_t *__restrict__ off,
                                                     const uint64_t *__restrict__ entries,
                                                     const unsigned long long *__restrict__ starts,
                                                     uint64_t *__restrict__ hits) {
    int pair, s;
    long long q0;
    query_item(qprefix, npairs, blockIdx.x, pair, s, q0);
    if (!((strands >> s) & 1)) return;
    const PairInfo P = pairs[pair];
    if ((long long)P.tlen < pat.span) return;
    const uint32_t *Qs = s ? Qrc : Q;
    const long long qb = s ? P.qoff_rc : P.qoff;
    const long long nq = (long long)P.qlen - pat.span + 1;
    for (long long q = q0 + threadIdx.x; q < min(nq, q0 + ITEM); q += BLOCK)
        bhits_at<true>(Qs, qb + q, q, P, pair, s, pat, transition, dbits, off, entries, hits,
                       starts[s * qtotal + P.qoff + q]);
}

// ---------------------------------------------------------------- one-pass hits

// One pass over the query side: each thread counts the hits of its query
// position, a warp reserves room for all of its lanes' hits with one atomic,
// and the hits are written there (the probes read again, now from L1/L2).
// Output order is not fixed; the caller sorts the hits by their whole word.
// Writes stop at `cap`; *total still counts every hit, so the caller can
// retry with enough room.
__global__ void __launch_bounds__(BLOCK) bhits_emit(const uint32_t *__restrict__ Q,
                                                    const uint32_t *__restrict__ Qrc,
                                                    const PairInfo *__restrict__ pairs,
                                                    const long long *__restrict__ qprefix,
                                                    int npairs, int strands, SeedPattern pat,
                                                    int transition, int dbits,
                                                    const uint32_t *__restrict__ off,
                                                    const uint64_t *__restrict__ entries,
                                                    unsigned long long *__restrict__ total,
                                                    unsigned long long cap,
                                                    uint64_t *__restrict__ hits) {
    int pair, s;
    long long q0;
    query_item(qprefix, npairs, blockIdx.x, pair, s, q0);
    if (!((strands >> s) & 1)) return;
    const PairInfo P = pairs[pair];
    if ((long long)P.tlen < pat.span) return;
    const uint32_t *Qs = s ? Qrc : Q;
    const long long qb = s ? P.qoff_rc : P.qoff;
    const long long nq = (long long)P.qlen - pat.span + 1;
    const int lane = threadIdx.x & 31;
    for (long long base = q0; base < min(nq, q0 + ITEM); base += BLOCK) {
        const long long q = base + threadIdx.x;
        const bool valid = q < min(nq, q0 + ITEM);
        const uint32_t c = valid ? bhits_at<false>(Qs, qb + q, q, P, pair, s, pat, transition,
                                                   dbits, off, entries, nullptr, 0)
                                 : 0u;
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        unsigned long long wbase = 0;
        const uint32_t wsum = __shfl_sync(0xffffffffu, incl, 31);
        if (lane == 31 && wsum) wbase = atomicAdd(total, (unsigned long long)wsum);
        wbase = __shfl_sync(0xffffffffu, wbase, 31);
        const unsigned long long o = wbase + incl - c;
        if (c && o + c <= cap)
            bhits_at<true>(Qs, qb + q, q, P, pair, s, pat, transition, dbits, off, entries, hits,
                           o);
    }
}

// ---------------------------------------------------------------- HSP order

__device__ __forceinline__ long long count_of(long long n, const unsigned long long *nd) {
    return nd ? min(n, (long long)*nd) : n;
}

__global__ void bhsp_keys(const BatchHsp *__restrict__ h, long long n,
                          const unsigned long long *nd, int lbits, uint64_t *__restrict__ keys,
                          unsigned *__restrict__ idx) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= count_of(n, nd)) return;
    const BatchHsp x = h[i];
    keys[i] = ((uint64_t)(uint32_t)x.pair << (2 * lbits + 1)) |
              ((uint64_t)(uint32_t)x.strand << (2 * lbits)) |
              ((uint64_t)(uint32_t)x.tpos << lbits) | (uint64_t)(uint32_t)x.qpos;
    idx[i] = (unsigned)i;
}

__global__ void bhsp_gather(const BatchHsp *__restrict__ h, const unsigned *__restrict__ idx,
                            long long n, const unsigned long long *nd,
                            BatchHsp *__restrict__ out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= count_of(n, nd)) return;
    out[i] = h[idx[i]];
}

__device__ __forceinline__ bool bhsp_less(const BatchHsp &a, const BatchHsp &b) {
    if (a.len != b.len) return a.len < b.len;
    return a.score < b.score;
}

// Runs of equal (pair, strand, tpos, qpos) ordered by (len, score).
__global__ void bhsp_fix_runs(BatchHsp *__restrict__ h, const uint64_t *__restrict__ keys,
                              long long n, const unsigned long long *nd) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    n = count_of(n, nd);
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

cudaError_t launch_batch_index(const uint32_t *T, const PairInfo *pairs, const long long *tprefix,
                               long long titems, int npairs, SeedPattern pat, uint32_t *cnt,
                               long long nbuckets, uint32_t *off, uint64_t *entries, void *tmp,
                               cudaStream_t st) {
    cudaMemsetAsync(cnt, 0, (size_t)nbuckets * 4, st);
    if (titems > 0) {
        g_launches++;
        bidx_count<<<(unsigned)titems, BLOCK, 0, st>>>(T, pairs, tprefix, npairs, pat, cnt);
    }
    cudaError_t e = scan_u32_to_u32(cnt, off, nbuckets, tmp, st);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(cnt, 0, (size_t)nbuckets * 4, st);  // reused as placement cursors
    if (titems > 0) {
        g_launches++;
        bidx_fill<<<(unsigned)titems, BLOCK, 0, st>>>(T, pairs, tprefix, npairs, pat, off, cnt,
                                                      entries);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_hit_count(const uint32_t *Q, const uint32_t *Qrc, const PairInfo *pairs,
                                   const long long *qprefix, long long qitems, int npairs,
                                   int strands_mask, SeedPattern pat, int transition, int dbits,
                                   long long qtotal, const uint32_t *off, const uint64_t *entries,
                                   uint32_t *counts, cudaStream_t st) {
    cudaMemsetAsync(counts, 0, (size_t)(2 * qtotal) * 4, st);
    if (qitems > 0) {
        g_launches++;
        bhits_count<<<(unsigned)qitems, BLOCK, 0, st>>>(Q, Qrc, pairs, qprefix, npairs,
                                                        strands_mask, pat, transition, dbits,
                                                        qtotal, off, entries, counts);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_hit_write(const uint32_t *Q, const uint32_t *Qrc, const PairInfo *pairs,
                                   const long long *qprefix, long long qitems, int npairs,
                                   int strands_mask, SeedPattern pat, int transition, int dbits,
                                   long long qtotal, const uint32_t *off, const uint64_t *entries,
                                   const unsigned long long *starts, uint64_t *hits,
                                   cudaStream_t st) {
    if (qitems > 0) {
        g_launches++;
        bhits_write<<<(unsigned)qitems, BLOCK, 0, st>>>(Q, Qrc, pairs, qprefix, npairs,
                                                        strands_mask, pat, transition, dbits,
                                                        qtotal, off, entries, starts, hits);
    }
    return cudaGetLastError();
}

int batch_item_size() { return ITEM; }

cudaError_t launch_batch_hit_emit(const uint32_t *Q, const uint32_t *Qrc, const PairInfo *pairs,
                                  const long long *qprefix, long long qitems, int npairs,
                                  int strands_mask, SeedPattern pat, int transition, int dbits,
                                  const uint32_t *off, const uint64_t *entries,
                                  unsigned long long *total, unsigned long long cap,
                                  uint64_t *hits, cudaStream_t st) {
    cudaMemsetAsync(total, 0, 8, st);
    if (qitems > 0) {
        g_launches++;
        bhits_emit<<<(unsigned)qitems, BLOCK, 0, st>>>(Q, Qrc, pairs, qprefix, npairs,
                                                       strands_mask, pat, transition, dbits, off,
                                                       entries, total, cap, hits);
    }
    return cudaGetLastError();
}



size_t batch_hsp_sort_temp_bytes(long long n) {
    n = n > 0 ? n : 1;
    return (size_t)n * (8 + 8 + 4 + 4 + sizeof(BatchHsp)) + radix_sort_temp_bytes(n) + 1536;
}

cudaError_t batch_hsp_sort(BatchHsp *h, long long n, const unsigned long long *nd, int pbits,
                           int lbits, void *tmp, BatchHsp **out, uint32_t *status,
                           cudaStream_t st) {
    *out = h;
    if (n <= 0 || (n <= 1 && !nd)) return cudaSuccess;
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
    bhsp_keys<<<grid_for(n), BLOCK, 0, st>>>(h, n, nd, lbits, ka, va);
    bool in_b = false;
    cudaError_t e = radix_sort_dev(ka, kb, va, vb, n, nd, 0, pbits + 1 + 2 * lbits, rt, &in_b,
                                   status, st);
    if (e != cudaSuccess) return e;
    uint64_t *kf = in_b ? kb : ka;
    unsigned *vf = in_b ? vb : va;
    g_launches += 2;
    bhsp_gather<<<grid_for(n), BLOCK, 0, st>>>(h, vf, n, nd, hb);
    bhsp_fix_runs<<<grid_for(n), BLOCK, 0, st>>>(hb, kf, n, nd);
    *out = hb;
    return cudaGetLastError();
}

}  // namespace sfe
