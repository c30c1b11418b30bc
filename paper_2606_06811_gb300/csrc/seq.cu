// Sequence kernels: 2-bit packing, reverse complement, spaced-seed keys, the
// CSR offsets of the seeding index, and hit-record conversions.
#include "sfe_internal.cuh"

namespace sfe {

namespace {

// ASCII -> code, 255 for anything outside ACGTacgt.
__device__ __forceinline__ uint32_t ascii_code(uint32_t c) {
    uint32_t u = c & 0xDFu;  // upper-case letters
    uint32_t code = ((u >> 1) ^ (u >> 2)) & 3u;  // A->0 C->1 G->2 T->3
    bool ok = (u == 'A' || u == 'C' || u == 'G' || u == 'T') && (c & 0x80u) == 0;
    return ok ? code : 255u;
}

// One packed word (16 bases) per thread, reading 16 input bytes with one
// 128-bit load when the whole word is inside the input and the input is
// 16-byte aligned.
__global__ void pack_kernel(const uint8_t *__restrict__ src, long long n, int codes,
                            uint32_t *__restrict__ dst, long long nwords,
                            uint32_t *__restrict__ status) {
    long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = nwords + 2 * SEQ_PAD;
    if (w >= total) return;
    long long word = w - SEQ_PAD;  // may be negative (front padding)
    uint32_t out = 0, bad = 0;
    if (word >= 0 && word < nwords) {
        long long b0 = word * 16;
        uint8_t bytes[16];
        bool aligned = ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) && (b0 + 16 <= n);
        if (aligned) {
            uint4 v = __ldg(reinterpret_cast<const uint4 *>(src + b0));
            *reinterpret_cast<uint4 *>(bytes) = v;
        } else {
#pragma unroll
            for (int i = 0; i < 16; i++) bytes[i] = (b0 + i < n) ? src[b0 + i] : (uint8_t)'A';
        }
        int m = (int)min(16LL, n - b0);
#pragma unroll
        for (int i = 0; i < 16; i++) {
            uint32_t c = bytes[i];
            uint32_t code = codes ? (c < 4u ? c : 255u) : ascii_code(c);
            if (i < m) {
                bad |= (code == 255u);
                out |= (code & 3u) << (2 * i);
            }
        }
    }
    dst[w - SEQ_PAD] = out;
    if (bad) atomicOr(status, ST_BAD_SYMBOL);
}

__device__ __forceinline__ uint32_t rev2(uint32_t x) {
    x = __brev(x);
    return ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);
}

// rc word j holds bases 16j..16j+15 of the reverse complement: the complement
// of bases n-1-16j .. n-16-16j of the forward sequence, in reverse order.
__global__ void revcomp_kernel(const uint32_t *__restrict__ src, long long n,
                               uint32_t *__restrict__ dst, long long nwords) {
    long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = nwords + 2 * SEQ_PAD;
    if (w >= total) return;
    long long j = w - SEQ_PAD;
    uint32_t out = 0;
    if (j >= 0 && j < nwords) {
        long long p0 = n - 16 - 16 * j;  // forward base that lands at rc position 16j+15
        uint32_t fw = win16(src, p0);
        out = ~rev2(fw);
        long long valid = n - 16 * j;  // rc bases present in this word
        if (valid < 16) out &= (1u << (2 * valid)) - 1u;
    }
    dst[w - SEQ_PAD] = out;
}

// Cell plane of a packed sequence of n bases (layout in WalkParams): word j
// holds bases 8j..8j+7 (one half of a 2-bit word spread to nibbles), each
// code shifted left by `shift`; bases past the end and the PLANE_PAD words on
// either side read as 0. dst is the base 0 pointer.
__device__ __forceinline__ uint32_t spread_nibbles(uint32_t x) {
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    return (x | (x << 2)) & 0x33333333u;
}

__global__ void plane_kernel(const uint32_t *__restrict__ S, long long n, int shift,
                             uint32_t *__restrict__ dst, long long nw) {
    const long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (w >= nw + 2 * PLANE_PAD) return;
    const long long j = w - PLANE_PAD;  // may be negative (front padding)
    uint32_t f = 0;
    if (j >= 0 && j < nw) {
        const long long p = 8 * j;
        const uint32_t h = (__ldg(S + (p >> 4)) >> (16 * ((p >> 3) & 1))) & 0xFFFFu;
        f = spread_nibbles(h) << shift;
        if (n - p < 8) f &= (1u << (4 * (n - p))) - 1u;
    }
    dst[j] = f;
}

__global__ void seed_keys_kernel(const uint32_t *__restrict__ S, long long nidx, SeedPattern pat,
                                 uint64_t *__restrict__ keys) {
    long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= nidx) return;
    const long long p = j * pat.step;
    uint64_t v = (uint64_t)win16(S, p) | ((uint64_t)win16(S, p + 16) << 32);
    uint32_t k = 0;
    for (int i = 0; i < pat.weight; i++) k = (k << 2) | (uint32_t)((v >> (2 * pat.care[i])) & 3u);
    keys[j] = ((uint64_t)k << 32) | (uint32_t)p;
}

// Bucket sizes of the CSR table (counts must be zeroed) and the positions
// column: counts[key(i)] += 1, positions[i] = low word of sorted[i].
__global__ void csr_count_kernel(const uint64_t *__restrict__ sorted, long long m,
                                 uint32_t *__restrict__ counts, uint32_t *__restrict__ positions,
                                 int shift, uint16_t *__restrict__ low) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint64_t v = sorted[i];
    positions[i] = (uint32_t)v;
    const uint32_t key = (uint32_t)(v >> 32);
    if (low) low[i] = (uint16_t)(key & ((1u << shift) - 1u));
    atomicAdd(counts + (key >> shift), 1u);
}

__global__ void hits_to_public_kernel(const uint64_t *__restrict__ hits, long long n, int strand,
                                      long long qoff, sfe_hit *__restrict__ out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t h = hits[i];
    long long D = (long long)((h >> 32) & 0x7FFFFFFFu);
    long long t = (long long)(uint32_t)h;
    sfe_hit r;
    r.strand = strand;
    r.tpos = (int32_t)t;
    r.qpos = (int32_t)(t - D + qoff);
    out[i] = r;
}

// Public record -> strand << 63 | D << 32 | t, with D = t - q + (qlen - span).
__global__ void public_to_walk_kernel(const sfe_hit *__restrict__ in, long long n, long long tlen,
                                      long long qlen, int span, uint64_t *__restrict__ out,
                                      uint32_t *__restrict__ status) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    sfe_hit h = in[i];
    bool ok = (h.strand == 0 || h.strand == 1) && h.tpos >= 0 && h.qpos >= 0 &&
              (long long)h.tpos + span <= tlen && (long long)h.qpos + span <= qlen;
    if (!ok) {
        atomicOr(status, ST_BAD_HIT);
        out[i] = 0;
        return;
    }
    long long D = (long long)h.tpos - h.qpos + (qlen - span);
    out[i] = ((uint64_t)(uint32_t)h.strand << 63) | ((uint64_t)D << 32) | (uint32_t)h.tpos;
}

inline unsigned grid_for(long long n, int block = BLOCK) {
    return (unsigned)((n + block - 1) / block);
}

}  // namespace

cudaError_t launch_pack(const uint8_t *src, long long n, int codes, uint32_t *dst,
                        uint32_t *status, cudaStream_t st) {
    long long nwords = (n + 15) / 16;
    long long total = nwords + 2 * SEQ_PAD;
    g_launches++;
    pack_kernel<<<grid_for(total), BLOCK, 0, st>>>(src, n, codes, dst, nwords, status);
    return cudaGetLastError();
}

cudaError_t launch_revcomp(const uint32_t *src, long long n, uint32_t *dst, cudaStream_t st) {
    long long nwords = (n + 15) / 16;
    long long total = nwords + 2 * SEQ_PAD;
    g_launches++;
    revcomp_kernel<<<grid_for(total), BLOCK, 0, st>>>(src, n, dst, nwords);
    return cudaGetLastError();
}

size_t plane_words(long long n) { return (size_t)((n + 7) / 8) + 2 * PLANE_PAD; }

cudaError_t launch_plane(const uint32_t *S, long long n, int shift, uint32_t *dst,
                         cudaStream_t st) {
    const long long nw = (n + 7) / 8;
    g_launches++;
    plane_kernel<<<grid_for(nw + 2 * PLANE_PAD), BLOCK, 0, st>>>(S, n, shift, dst, nw);
    return cudaGetLastError();
}

cudaError_t launch_seed_keys(const uint32_t *S, long long n, SeedPattern pat, uint64_t *keys,
                             cudaStream_t st) {
    const long long nidx = indexed_positions(pat, n);
    if (nidx <= 0) return cudaSuccess;
    g_launches++;
    seed_keys_kernel<<<grid_for(nidx), BLOCK, 0, st>>>(S, nidx, pat, keys);
    return cudaGetLastError();
}

cudaError_t launch_csr_counts(const uint64_t *sorted, long long m, uint32_t *counts,
                             uint32_t *positions, int shift, uint16_t *low, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    g_launches++;
    csr_count_kernel<<<grid_for(m), BLOCK, 0, st>>>(sorted, m, counts, positions, shift, low);
    return cudaGetLastError();
}

cudaError_t launch_hits_to_public(const uint64_t *hits, long long n, int strand, long long qoff,
                                  sfe_hit *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    g_launches++;
    hits_to_public_kernel<<<grid_for(n), BLOCK, 0, st>>>(hits, n, strand, qoff, out);
    return cudaGetLastError();
}

cudaError_t launch_public_to_walk(const sfe_hit *in, long long n, long long tlen, long long qlen,
                                  int span, uint64_t *out, uint32_t *status, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    g_launches++;
    public_to_walk_kernel<<<grid_for(n), BLOCK, 0, st>>>(in, n, tlen, qlen, span, out, status);
    return cudaGetLastError();
}

}  // namespace sfe
