// Seeding and HSP ordering for a batch of target/query pairs.
//
// Every pair has its own seeding index, so no hit ever joins two pairs.
//
// Two probes per query position instead of 1 + weight. A hit allows at most
// one transition among the care positions, and a transition keeps a base's
// purine/pyrimidine class (the low bit of the 2-bit code), so split the care
// positions into a first half A and a second half B: a hit has A exact, or B
// exact with the transition in A. Table 1 is keyed by (A's bases, B's
// classes), table 2 by (B's bases, A's classes). A probe of table 1 keeps the
// entries with A exact, all classes equal and at most one transition in B; a
// probe of table 2 keeps those with B exact, all classes equal and exactly one
// transition in A. Each hit is found once. Without transitions only table 1
// is probed, for exact keys.
//
// A pair with n seed positions gets 2^b buckets per table, b = ceil(log2 n)
// clamped to [4, table key bits], addressed by the top b bits of the table
// key; the buckets of all pairs sit back to back, table 2's after table 1's,
// in one CSR. Entries keep their full seed key and are checked against the
// probe's. The tables are filled by a counting sort (counts whose atomics also
// give each entry its place in its bucket, one exclusive scan over all
// buckets, then placement without atomics): the order inside a bucket is not
// fixed, and it need not be, because the hits are sorted by their whole word
// before the walk.
//
// Hit words: pair << (dbits + 1) | strand << dbits | local diagonal in the
// high half, local t in the low half.
#include "sfe_internal.cuh"

namespace sfe {

namespace {


// Halves of the care positions: A = the first weight / 2 (the key's high
// groups), B = the rest (its low groups). Table keys are left-aligned to
// split_bits() bits.
struct Split {
    int hA, hB, ik;          // sizes, table key width
    uint32_t maskB;          // B's groups in a seed key
    uint32_t low, highA, highB;  // class bits; transition bits of A and of B
};

__host__ __device__ __forceinline__ Split split_of(int weight) {
    Split q;
    q.hA = weight / 2;
    q.hB = weight - q.hA;
    q.ik = 2 * q.hB + q.hA;  // the wider of 2hA + hB and 2hB + hA
    q.maskB = (1u << (2 * q.hB)) - 1u;
    const uint32_t all = (weight >= 16) ? 0xFFFFFFFFu : ((1u << (2 * weight)) - 1u);
    q.low = 0x55555555u & all;
    q.highB = 0xAAAAAAAAu & q.maskB;
    q.highA = 0xAAAAAAAAu & all & ~q.maskB;
    return q;
}

// The class bits (low bit of each 2-bit group) of the n <= 8 groups of x, packed.
__device__ __forceinline__ uint32_t classes(uint32_t x) {
    x &= 0x5555u;
    x = (x | (x >> 1)) & 0x3333u;
    x = (x | (x >> 2)) & 0x0F0Fu;
    return (x | (x >> 4)) & 0x00FFu;
}

__device__ __forceinline__ uint32_t table1_key(uint32_t k, const Split &q) {
    const uint32_t key = ((k >> (2 * q.hB)) << q.hB) | classes(k & q.maskB);
    return key << (q.ik - (2 * q.hA + q.hB));
}

__device__ __forceinline__ uint32_t table2_key(uint32_t k, const Split &q) {
    return ((k & q.maskB) << q.hA) | classes(k >> (2 * q.hB));
}

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
                                                    int npairs, SeedPattern pat, long long nb,
                                                    uint32_t *__restrict__ cnt,
                                                    uint2 *__restrict__ slots) {
    const int p = item_pair(tprefix, npairs, blockIdx.x);
    const PairInfo P = pairs[p];
    const long long npos = (long long)P.tlen - pat.span + 1;
    const long long i0 = (blockIdx.x - tprefix[p]) * (long long)ITEM;
    const Split q = split_of(pat.weight);
    for (long long i = i0 + threadIdx.x; i < min(npos, i0 + ITEM); i += BLOCK) {
        if (i % pat.step) continue;  // the index stride: only every step-th position
        const uint32_t k = spaced_key(T, P.toff + i, pat);
        uint2 sl;
        sl.x = atomicAdd(cnt + P.boff + (table1_key(k, q) >> (q.ik - P.bbits)), 1u);
        sl.y = atomicAdd(cnt + nb + P.boff + (table2_key(k, q) >> (q.ik - P.bbits)), 1u);
        slots[P.toff + i] = sl;  // the entry's place in each bucket, used by the fill
    }
}

// Entries (key << 32 | local position) in their buckets, one work item per block.
__global__ void __launch_bounds__(BLOCK) bidx_fill(const uint32_t *__restrict__ T,
                                                   const PairInfo *__restrict__ pairs,
                                                   const long long *__restrict__ tprefix,
                                                   int npairs, SeedPattern pat, long long nb,
                                                   const uint32_t *__restrict__ off,
                                                   const uint2 *__restrict__ slots,
                                                   uint64_t *__restrict__ entries) {
    const int p = item_pair(tprefix, npairs, blockIdx.x);
    const PairInfo P = pairs[p];
    const long long npos = (long long)P.tlen - pat.span + 1;
    const long long i0 = (blockIdx.x - tprefix[p]) * (long long)ITEM;
    const Split q = split_of(pat.weight);
    for (long long i = i0 + threadIdx.x; i < min(npos, i0 + ITEM); i += BLOCK) {
        if (i % pat.step) continue;
        const uint32_t k = spaced_key(T, P.toff + i, pat);
        const uint64_t ent = ((uint64_t)k << 32) | (uint32_t)i;
        const uint2 sl = slots[P.toff + i];
        entries[off[P.boff + (table1_key(k, q) >> (q.ik - P.bbits))] + sl.x] = ent;
        entries[off[nb + P.boff + (table2_key(k, q) >> (q.ik - P.bbits))] + sl.y] = ent;
    }
}

// Hits of query position q (pair P, strand s) against P's tables. The probe
// (seed key, the two buckets' bounds, the hit word's fixed part) is made once;
// the buckets are scanned once to count the entries their tables accept and,
// for a position with hits, once more to write them from `o` on.
struct BProbe {
    uint32_t k, a1, e1, a2, e2, hi_base;
    long long dq;  // D = t + dq
};

__device__ __forceinline__ BProbe bprobe(const uint32_t *__restrict__ Qs, long long qg,
                                         long long q, const PairInfo &P, int pair, int s,
                                         const SeedPattern &pat, int transition, int dbits,
                                         long long nb, const uint32_t *__restrict__ off) {
    BProbe b;
    b.k = spaced_key(Qs, qg, pat);
    const Split sp = split_of(pat.weight);
    const long long b1 = P.boff + (table1_key(b.k, sp) >> (sp.ik - P.bbits));
    const long long b2 = nb + P.boff + (table2_key(b.k, sp) >> (sp.ik - P.bbits));
    b.a1 = __ldg(off + b1);
    b.e1 = __ldg(off + b1 + 1);
    b.a2 = transition ? __ldg(off + b2) : 0u;
    b.e2 = transition ? __ldg(off + b2 + 1) : 0u;
    b.hi_base = ((uint32_t)pair << (dbits + 1)) | ((uint32_t)s << dbits);
    b.dq = (long long)P.qlen - pat.span - q;
    return b;
}

template <bool WRITE>
__device__ __forceinline__ uint32_t bhits_scan(const BProbe &b, const SeedPattern &pat,
                                               int transition,
                                               const uint64_t *__restrict__ entries,
                                               uint64_t *__restrict__ out, unsigned long long o) {
    const Split sp = split_of(pat.weight);
    uint32_t c = 0;
    for (uint32_t j = b.a1; j < b.e1; j++) {
        const uint64_t ent = __ldg(entries + j);
        const uint32_t x = (uint32_t)(ent >> 32) ^ b.k;
        // A exact, classes equal, at most one transition in B (none without transitions)
        const bool hit = transition ? ((x & (sp.low | sp.highA)) == 0 && __popc(x & sp.highB) <= 1)
                                    : x == 0;
        if (!hit) continue;
        if (WRITE) {
            const uint32_t t = (uint32_t)ent;
            out[o + c] = ((uint64_t)(b.hi_base | (uint32_t)(t + b.dq)) << 32) | t;
        }
        c++;
    }
    for (uint32_t j = b.a2; j < b.e2; j++) {
        const uint64_t ent = __ldg(entries + j);
        const uint32_t x = (uint32_t)(ent >> 32) ^ b.k;
        // B exact, classes equal, exactly one transition in A
        if ((x & (sp.low | sp.highB)) != 0 || __popc(x & sp.highA) != 1) continue;
        if (WRITE) {
            const uint32_t t = (uint32_t)ent;
            out[o + c] = ((uint64_t)(b.hi_base | (uint32_t)(t + b.dq)) << 32) | t;
        }
        c++;
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

// ---------------------------------------------------------------- one-pass hits

// One pass over the query side: each thread counts the hits of its query
// position, a warp reserves room for all of its lanes' hits with one atomic,
// and the hits are written there (the probe's buckets scanned again, now from
// L1/L2; the probe itself is kept in registers: recomputing it for the few
// positions with hits ran the whole probe path with one or two lanes of a
// warp active).
// Output order is not fixed; the caller sorts the hits by their whole word.
// Writes stop at `cap`; *total still counts every hit, so the caller can
// retry with enough room.
__global__ void __launch_bounds__(BLOCK) bhits_emit(const uint32_t *__restrict__ Q,
                                                    const uint32_t *__restrict__ Qrc,
                                                    const PairInfo *__restrict__ pairs,
                                                    const long long *__restrict__ qprefix,
                                                    int npairs, int strands, SeedPattern pat,
                                                    int transition, int dbits, long long nb,
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
        BProbe pr{};
        if (valid) pr = bprobe(Qs, qb + q, q, P, pair, s, pat, transition, dbits, nb, off);
        const uint32_t c = valid ? bhits_scan<false>(pr, pat, transition, entries, nullptr, 0) : 0u;
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
        if (c && o + c <= cap) bhits_scan<true>(pr, pat, transition, entries, hits, o);
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
                               long long nbuckets, uint32_t *off, uint64_t *entries, uint2 *slots,
                               void *tmp, cudaStream_t st) {
    const long long nb2 = 2 * nbuckets;  // both tables
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)nb2 * 4, st);
    if (e != cudaSuccess) return e;
    if (titems > 0) {
        g_launches++;
        bidx_count<<<(unsigned)titems, BLOCK, 0, st>>>(T, pairs, tprefix, npairs, pat, nbuckets,
                                                       cnt, slots);
    }
    e = scan_u32_to_u32(cnt, off, nb2, tmp, st);
    if (e != cudaSuccess) return e;
    if (titems > 0) {
        g_launches++;
        bidx_fill<<<(unsigned)titems, BLOCK, 0, st>>>(T, pairs, tprefix, npairs, pat, nbuckets,
                                                      off, slots, entries);
    }
    return cudaGetLastError();
}

int batch_table_bits(int weight) { return split_of(weight).ik; }

int batch_item_size() { return ITEM; }

cudaError_t launch_batch_hit_emit(const uint32_t *Q, const uint32_t *Qrc, const PairInfo *pairs,
                                  const long long *qprefix, long long qitems, int npairs,
                                  int strands_mask, SeedPattern pat, int transition, int dbits,
                                  long long nbuckets, const uint32_t *off,
                                  const uint64_t *entries, unsigned long long *total,
                                  unsigned long long cap, uint64_t *hits, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(total, 0, 8, st);
    if (e != cudaSuccess) return e;
    if (qitems > 0) {
        g_launches++;
        bhits_emit<<<(unsigned)qitems, BLOCK, 0, st>>>(Q, Qrc, pairs, qprefix, npairs,
                                                       strands_mask, pat, transition, dbits,
                                                       nbuckets, off, entries, total, cap, hits);
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
