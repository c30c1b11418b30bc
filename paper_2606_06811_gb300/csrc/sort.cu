// Device radix sort (stable, LSD, 8-bit digits), exclusive scans and the HSP
// ordering. Written from scratch: no CUB in the library.
//
// Radix sort per 8-bit digit pass, over a grid of G CTAs that each own one
// contiguous chunk of the input (a whole number of 4096-element tiles):
//   1. rs_hist:    per-CTA digit counts -> counts[digit * G + cta], digit totals
//   2. rs_offsets: per digit, exclusive scan over CTAs plus the digit's base
//   3. rs_scatter: each CTA walks its tiles in order; the next tile's keys
//      arrive by one bulk asynchronous copy (TMA, cp.async.bulk completing on
//      an mbarrier) while the current one is ranked; warps rank their elements
//      stably with __match_any_sync in element order, the tile is reordered in
//      shared memory, and runs of equal digits are written out contiguously.
//      (The bulk copy replaced per-thread 16-byte cp.async copies: hit sort of
//      the 10 Mb pair 5.11 against 5.21 ms per step. The per-warp digit counts
//      are packed two to a word, which halves the clearing and the cross-warp
//      prefix of every tile: 5.04 against 5.10 ms. Packing each key's digit
//      and rank into one register as well removed the last spills but was
//      slower, 5.13 ms.)
// Traffic per pass: the keys are read twice and written once (plus values).
#include "sfe_internal.cuh"

namespace sfe {

namespace {

// 256 threads x 16 keys per tile: measured against 256 x 8, 512 x 8, 512 x 16
// and 128 x 32 on the 10 Mb pair's hit sort (5.5 ms against 5.9-7.3 ms).
constexpr int RS_BLOCK = 256;
constexpr int RS_WARPS = RS_BLOCK / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_BLOCK * RS_ITEMS;  // 4096
// Digits of up to 9 bits (512 buckets); 10 bits (1024) only where that saves a
// pass, since the wider histograms cost every tile more (measured: a 25-bit
// key sorts faster with 512 buckets than with 1024, a 28-bit key faster in
// three passes of up to 10 bits than in four of 7).
constexpr int RS_MAXBITS = 10;
constexpr int RS_R = 1 << RS_MAXBITS;  // largest bucket count (sizes the count arrays)

int num_sms() { return device_sms(); }

struct RsGeom {
    int G;
    long long chunk;
};

RsGeom rs_geom(long long n) {
    long long tiles = (n + RS_TILE - 1) / RS_TILE;
    long long gmax = 4LL * num_sms();
    long long G = tiles < gmax ? tiles : gmax;
    if (G < 1) G = 1;
    long long per = (tiles + G - 1) / G;
    RsGeom g;
    g.G = (int)((tiles + per - 1) / per);
    if (g.G < 1) g.G = 1;
    g.chunk = per * RS_TILE;
    return g;
}

// With a device count `nd`, n is the capacity the grid was sized for and each
// CTA derives the key count and its chunk from *nd.
__device__ __forceinline__ void rs_device_count(const unsigned long long *nd, int G, long long &n,
                                                long long &chunk) {
    if (!nd) return;
    n = min(n, (long long)*nd);
    const long long tiles = (n + RS_TILE - 1) / RS_TILE;
    chunk = max(1LL, (tiles + G - 1) / G) * RS_TILE;
}

// DEVN: the key count is read from *nd (a separate instantiation, so the
// host-count kernels keep their parameters in the constant bank)
template <int R, bool DEVN>
__global__ void __launch_bounds__(RS_BLOCK) rs_hist(const uint64_t *__restrict__ keys,
                                                    long long n, const unsigned long long *nd,
                                                    int shift, unsigned mask, long long chunk,
                                                    unsigned *__restrict__ counts,
                                                    unsigned *__restrict__ totals, int G) {
    __shared__ unsigned h[RS_WARPS][R];
    if (DEVN) rs_device_count(nd, G, n, chunk);
    for (int i = threadIdx.x; i < RS_WARPS * R; i += RS_BLOCK) (&h[0][0])[i] = 0;
    __syncthreads();
    long long beg = (long long)blockIdx.x * chunk;
    long long end = min(n, beg + chunk);
    int w = threadIdx.x >> 5;
    for (long long i = beg + threadIdx.x; i < end; i += RS_BLOCK) {
        unsigned d = (unsigned)(keys[i] >> shift) & mask;
        atomicAdd(&h[w][d], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < R; d += RS_BLOCK) {
        unsigned s = 0;
#pragma unroll
        for (int k = 0; k < RS_WARPS; k++) s += h[k][d];
        counts[(long long)d * G + blockIdx.x] = s;
        if (s) atomicAdd(&totals[d], s);
    }
}

// Inclusive warp scan.
__device__ __forceinline__ unsigned warp_incl(unsigned v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_incl64(unsigned long long v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Exclusive scan over a block of BLOCK threads (one value each); returns the
// thread's exclusive prefix and the block total in *total. Uses `sh` (>= 33).
template <int NT>
__device__ __forceinline__ unsigned long long block_excl64(unsigned long long v,
                                                           unsigned long long *sh,
                                                           unsigned long long *total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long inc = warp_incl64(v);
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    if (w == 0) {
        unsigned long long s = (lane < NT / 32) ? sh[lane] : 0ull;
        unsigned long long si = warp_incl64(s);
        if (lane < NT / 32) sh[lane] = si - s;
        if (lane == 31) sh[32] = si;
    }
    __syncthreads();
    unsigned long long r = sh[w] + inc - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

// Block d: offsets[d * G + g] = sum(totals[< d]) + sum(counts[d * G + < g]).
__global__ void __launch_bounds__(RS_BLOCK) rs_offsets(unsigned *__restrict__ counts,
                                                       const unsigned *__restrict__ totals, int G) {
    __shared__ unsigned long long sh[33];
    int d = blockIdx.x;
    unsigned long long b = 0;
    for (int k = threadIdx.x; k < d; k += RS_BLOCK) b += totals[k];
    unsigned long long tot;
    block_excl64<RS_BLOCK>(b, sh, &tot);
    unsigned long long carry = tot;
    for (int base = 0; base < G; base += RS_BLOCK) {
        int g = base + threadIdx.x;
        unsigned long long c = (g < G) ? counts[(long long)d * G + g] : 0ull;
        unsigned long long t2;
        unsigned long long ex = block_excl64<RS_BLOCK>(c, sh, &t2);
        if (g < G) counts[(long long)d * G + g] = (unsigned)(carry + ex);
        carry += t2;
    }
}

// Asynchronous copy of a tile's keys (count <= RS_TILE) into shared memory,
// 16 bytes per copy, the ragged end zero-filled; the scatter issues it for
// the next tile while it ranks and writes the current one. The keys must be
// 16-byte aligned (checked by the host).
__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// One bulk asynchronous copy (TMA, 1-D) of a tile's keys into shared memory,
// completing on the mbarrier: thread 0 issues it; an odd last key is copied
// by hand after the wait (a bulk copy moves multiples of 16 bytes).
__device__ __forceinline__ void rs_prefetch(uint64_t *dst, const uint64_t *src, unsigned count,
                                            uint64_t *mbar) {
    if (threadIdx.x == 0) {
        const unsigned bytes = (count * 8u) & ~15u;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
                     "r"(bytes)
                     : "memory");
        if (bytes)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                "[%3];" ::"r"(smem_u32(dst)),
                "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                : "memory");
    }
}

// Bounded wait for the tile's copy; false after about 2^26 polls.
__device__ __forceinline__ bool rs_wait(uint64_t *mbar, unsigned parity) {
    for (long long spins = 0; spins < (1LL << 26); spins++) {
        unsigned done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, "
            "0, p; }"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <bool VALS, int R, bool DEVN>
__global__ void __launch_bounds__(RS_BLOCK, 2) rs_scatter(
    const uint64_t *__restrict__ kin, uint64_t *__restrict__ kout,
    const unsigned *__restrict__ vin, unsigned *__restrict__ vout, long long n,
    const unsigned long long *nd, int shift, unsigned mask, long long chunk,
    const unsigned *__restrict__ offsets, int G, uint32_t *status) {
    if (DEVN) rs_device_count(nd, G, n, chunk);
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sraw = reinterpret_cast<uint64_t *>(smem);                   // RS_TILE: next tile
    uint64_t *sk = sraw + RS_TILE;                                          // RS_TILE
    unsigned *sv = reinterpret_cast<unsigned *>(sk + RS_TILE);              // RS_TILE (VALS)
    // per-warp digit counts, two 16-bit counts per word (a warp counts at most
    // 512 keys of a digit and the 8 warps of a tile at most 4096, so neither
    // half carries into the other)
    constexpr int RW = (R + 2) / 2;                                         // words per warp
    unsigned *wh = sv + (VALS ? RS_TILE : 0);                               // RS_WARPS*RW
    unsigned *tcount = wh + RS_WARPS * RW;                                  // R+1
    unsigned *tstart = tcount + (R + 1);                                 // R+1
    unsigned *run = tstart + (R + 1);                                    // R

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const long long beg = (long long)blockIdx.x * chunk;
    const long long end = min(n, beg + chunk);
    __shared__ __align__(8) uint64_t mbar;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned parity = 0;
    for (int d = tid; d < R; d += RS_BLOCK) run[d] = offsets[(long long)d * G + blockIdx.x];
    if (beg < end) rs_prefetch(sraw, kin + beg, (unsigned)min((long long)RS_TILE, end - beg), &mbar);

    for (long long tb = beg; tb < end; tb += RS_TILE) {
        const unsigned tile_n = (unsigned)min((long long)RS_TILE, end - tb);
        for (int i = tid; i < RS_WARPS * RW; i += RS_BLOCK) wh[i] = 0;
        if (!rs_wait(&mbar, parity)) {  // never on valid memory; bounded all the same
            if (tid == 0 && status) atomicOr(status, ST_TIMEOUT);
            rs_wait(&mbar, parity);  // the copy in flight, once more (bounded) before leaving
            return;
        }
        parity ^= 1u;
        if (tid == 0 && (tile_n & 1u)) sraw[tile_n - 1] = kin[tb + tile_n - 1];
        __syncthreads();

        uint64_t k[RS_ITEMS];
        unsigned v[RS_ITEMS], dg[RS_ITEMS], rk[RS_ITEMS];
        const unsigned wbase = w * 32 * RS_ITEMS;
#pragma unroll
        for (int j = 0; j < RS_ITEMS; j++) {
            unsigned e = wbase + j * 32 + lane;
            bool valid = e < tile_n;
            k[j] = valid ? sraw[e] : ~0ull;
            if (VALS) v[j] = valid ? vin[tb + e] : 0u;
            dg[j] = valid ? ((unsigned)(k[j] >> shift) & mask) : (unsigned)R;
        }
        __syncthreads();  // every thread has its keys: the buffer takes the next tile
        if (tb + RS_TILE < end)
            rs_prefetch(sraw, kin + tb + RS_TILE,
                        (unsigned)min((long long)RS_TILE, end - (tb + RS_TILE)), &mbar);
        unsigned *myh = wh + w * RW;
#pragma unroll
        for (int j = 0; j < RS_ITEMS; j++) {
            // the digit's lowest lane adds the group's size and shares the old
            // count; the next item's atomics follow this item's shuffle, so
            // the ranks keep the item order (a stable ranking)
            const unsigned peers = __match_any_sync(0xffffffffu, dg[j]);
            const int leader = __ffs(peers) - 1;
            const unsigned hs = (dg[j] & 1u) * 16u;
            unsigned old = 0;
            if (lane == leader) old = atomicAdd(myh + (dg[j] >> 1), (unsigned)__popc(peers) << hs);
            old = (__shfl_sync(0xffffffffu, old, leader) >> hs) & 0xFFFFu;
            rk[j] = old + __popc(peers & ((1u << lane) - 1u));
        }
        __syncwarp();
        __syncthreads();
        // per digit: exclusive prefix across warps, tile totals
        for (int d2 = tid; d2 < RW; d2 += RS_BLOCK) {
            unsigned s = 0;
#pragma unroll
            for (int ww = 0; ww < RS_WARPS; ww++) {
                unsigned c = wh[ww * RW + d2];
                wh[ww * RW + d2] = s;
                s += c;
            }
            tcount[2 * d2] = s & 0xFFFFu;
            if (2 * d2 + 1 <= R) tcount[2 * d2 + 1] = s >> 16;
        }
        __syncthreads();
        // exclusive scan of tcount[0..R] by warp 0 (17 values per lane)
        if (w == 0) {
            constexpr int PER = (R + 1 + 31) / 32;
            unsigned loc[PER], s = 0;
#pragma unroll
            for (int i = 0; i < PER; i++) {
                int d = lane * PER + i;
                loc[i] = (d <= R) ? tcount[d] : 0u;
                s += loc[i];
            }
            unsigned inc = warp_incl(s);
            unsigned ex = inc - s;
#pragma unroll
            for (int i = 0; i < PER; i++) {
                int d = lane * PER + i;
                if (d <= R) tstart[d] = ex;
                ex += loc[i];
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < RS_ITEMS; j++) {
            unsigned pos = tstart[dg[j]] + ((myh[dg[j] >> 1] >> ((dg[j] & 1u) * 16u)) & 0xFFFFu) +
                           rk[j];
            sk[pos] = k[j];
            if (VALS) sv[pos] = v[j];
        }
        __syncthreads();
        for (unsigned p = tid; p < tile_n; p += RS_BLOCK) {
            uint64_t kk = sk[p];
            unsigned d = (unsigned)(kk >> shift) & mask;
            unsigned o = run[d] + (p - tstart[d]);
            kout[o] = kk;
            if (VALS) vout[o] = sv[p];
        }
        __syncthreads();
        for (int d = tid; d < R; d += RS_BLOCK) run[d] += tcount[d];
        __syncthreads();
    }
}

size_t rs_smem(bool vals, int R) {
    return 2 * (size_t)RS_TILE * 8 + (vals ? (size_t)RS_TILE * 4 : 0) +
           (size_t)RS_WARPS * ((R + 2) / 2) * 4 + 2 * (size_t)(R + 1) * 4 + (size_t)R * 4;
}

// One LSD pass with 2^bits <= R buckets.
template <int R, bool DEVN>
cudaError_t rs_pass(const uint64_t *kin, uint64_t *kout, const uint32_t *vin, uint32_t *vout,
                    long long n, const unsigned long long *nd, int shift, unsigned mask,
                    const RsGeom &g, unsigned *counts, unsigned *totals, uint32_t *status,
                    cudaStream_t st) {
    const bool vals = vin != nullptr;
    const size_t smem = rs_smem(vals, R);
    static std::atomic<unsigned long long> attr_set[2];
    cudaError_t ae = once_per_device(attr_set[vals], [&] {
        return vals ? cudaFuncSetAttribute(rs_scatter<true, R, DEVN>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                    : cudaFuncSetAttribute(rs_scatter<false, R, DEVN>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (ae != cudaSuccess) return ae;
    cudaError_t me = cudaMemsetAsync(totals, 0, R * 4, st);
    if (me != cudaSuccess) return me;
    g_launches += 3;
    rs_hist<R, DEVN><<<g.G, RS_BLOCK, 0, st>>>(kin, n, nd, shift, mask, g.chunk, counts, totals,
                                               g.G);
    rs_offsets<<<R, RS_BLOCK, 0, st>>>(counts, totals, g.G);
    if (vals)
        rs_scatter<true, R, DEVN><<<g.G, RS_BLOCK, smem, st>>>(kin, kout, vin, vout, n, nd, shift,
                                                               mask, g.chunk, counts, g.G, status);
    else
        rs_scatter<false, R, DEVN><<<g.G, RS_BLOCK, smem, st>>>(kin, kout, nullptr, nullptr, n,
                                                                nd, shift, mask, g.chunk, counts,
                                                                g.G, status);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- scans

constexpr int SC_BLOCK = 256;
constexpr int SC_ITEMS = 16;
constexpr long long SC_CHUNK = (long long)SC_BLOCK * SC_ITEMS;

template <typename Tin>
__global__ void __launch_bounds__(SC_BLOCK) scan_reduce(const Tin *__restrict__ in, long long n,
                                                        unsigned long long *__restrict__ part) {
    __shared__ unsigned long long sh[33];
    long long beg = (long long)blockIdx.x * SC_CHUNK;
    long long end = min(n, beg + SC_CHUNK);
    unsigned long long s = 0;
    for (long long i = beg + threadIdx.x; i < end; i += SC_BLOCK) s += in[i];
    unsigned long long tot;
    block_excl64<SC_BLOCK>(s, sh, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Exclusive scan of part[0..nb) in place, part[nb] = total. One block.
__global__ void __launch_bounds__(1024) scan_partials(unsigned long long *part, long long nb) {
    __shared__ unsigned long long sh[33];
    unsigned long long carry = 0;
    for (long long base = 0; base < nb; base += 1024) {
        long long i = base + threadIdx.x;
        unsigned long long v = i < nb ? part[i] : 0ull;
        unsigned long long tot;
        unsigned long long ex = block_excl64<1024>(v, sh, &tot);
        if (i < nb) part[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) part[nb] = carry;
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(SC_BLOCK) scan_down(const Tin *__restrict__ in,
                                                      Tout *__restrict__ out, long long n,
                                                      const unsigned long long *__restrict__ part,
                                                      long long nb) {
    __shared__ unsigned long long sh[33];
    long long beg = (long long)blockIdx.x * SC_CHUNK;
    long long end = min(n, beg + SC_CHUNK);
    unsigned long long carry = part[blockIdx.x];
    for (long long base = beg; base < end; base += SC_BLOCK) {
        long long i = base + threadIdx.x;
        unsigned long long v = i < end ? (unsigned long long)in[i] : 0ull;
        unsigned long long tot;
        unsigned long long ex = block_excl64<SC_BLOCK>(v, sh, &tot);
        if (i < end) out[i] = (Tout)(carry + ex);
        carry += tot;
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = (Tout)part[nb];
}

template <typename Tin, typename Tout>
cudaError_t scan_impl(const Tin *in, Tout *out, long long n, void *tmp, cudaStream_t st) {
    long long nb = (n + SC_CHUNK - 1) / SC_CHUNK;
    unsigned long long *part = reinterpret_cast<unsigned long long *>(tmp);
    if (n == 0) {
        cudaMemsetAsync(out, 0, sizeof(Tout), st);
        return cudaGetLastError();
    }
    g_launches += 3;
    scan_reduce<Tin><<<(unsigned)nb, SC_BLOCK, 0, st>>>(in, n, part);
    scan_partials<<<1, 1024, 0, st>>>(part, nb);
    scan_down<Tin, Tout><<<(unsigned)nb, SC_BLOCK, 0, st>>>(in, out, n, part, nb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- HSP sort

__global__ void hsp_keys(const Hsp *__restrict__ h, long long n, int qbits, uint64_t *keys,
                         unsigned *idx) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Hsp x = h[i];
    keys[i] = ((uint64_t)(uint32_t)x.strand << 62) | ((uint64_t)(uint32_t)x.tpos << qbits) |
              (uint64_t)(uint32_t)x.qpos;
    idx[i] = (unsigned)i;
}

__global__ void hsp_gather(const Hsp *__restrict__ h, const unsigned *__restrict__ idx,
                           long long n, Hsp *__restrict__ out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = h[idx[i]];
}

__device__ __forceinline__ bool hsp_less(const Hsp &a, const Hsp &b) {
    if (a.len != b.len) return a.len < b.len;
    return a.score < b.score;
}

// Runs of equal (strand, tpos, qpos) are ordered by (len, score); such runs
// are short (they need two HSPs that start at the same cell), so each run is
// insertion-sorted by the thread at its head.
__global__ void hsp_fix_runs(Hsp *__restrict__ h, const uint64_t *__restrict__ keys, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i > 0 && keys[i - 1] == keys[i]) return;
    long long j = i + 1;
    while (j < n && keys[j] == keys[i]) j++;
    for (long long a = i + 1; a < j; a++) {
        Hsp x = h[a];
        long long b = a - 1;
        while (b >= i && hsp_less(x, h[b])) {
            h[b + 1] = h[b];
            b--;
        }
        h[b + 1] = x;
    }
}

unsigned grid_for(long long n, int block = BLOCK) { return (unsigned)((n + block - 1) / block); }

}  // namespace

size_t radix_sort_temp_bytes(long long n) {
    RsGeom g = rs_geom(n > 0 ? n : 1);
    return (size_t)RS_R * g.G * 4 + RS_R * 4 + 256;
}

cudaError_t radix_sort(uint64_t *keys_a, uint64_t *keys_b, uint32_t *vals_a, uint32_t *vals_b,
                       long long n, int lo, int hi, void *tmp, bool *result_in_b, uint32_t *status,
                       cudaStream_t st) {
    return radix_sort_dev(keys_a, keys_b, vals_a, vals_b, n, nullptr, lo, hi, tmp, result_in_b,
                          status, st);
}

cudaError_t radix_sort_dev(uint64_t *keys_a, uint64_t *keys_b, uint32_t *vals_a, uint32_t *vals_b,
                           long long n, const unsigned long long *nd, int lo, int hi, void *tmp,
                           bool *result_in_b, uint32_t *status, cudaStream_t st) {
    // status receives ST_TIMEOUT if a tile's bulk copy never completed (a
    // bounded wait that valid memory never runs out)
    *result_in_b = false;
    if (hi <= lo || n <= 0 || (n <= 1 && !nd)) return cudaSuccess;
    if (n >= (1LL << 32)) return cudaErrorInvalidValue;
    // the scatter copies keys 16 bytes at a time
    if ((reinterpret_cast<uintptr_t>(keys_a) | reinterpret_cast<uintptr_t>(keys_b)) & 15)
        return cudaErrorInvalidValue;
    RsGeom g = rs_geom(n);
    unsigned *counts = reinterpret_cast<unsigned *>(tmp);
    unsigned *totals = counts + (size_t)RS_R * g.G;
    // as few passes as 9-bit digits allow, or 10-bit ones where that saves a
    // pass, with the bits spread evenly (25 bits: 9 + 9 + 7; 28: 10 + 10 + 8)
    const int nbits = hi - lo;
    const int p9 = (nbits + 8) / 9, p10 = (nbits + 9) / 10;
    const int npass = p10 < p9 ? p10 : p9;
    const int per = (nbits + npass - 1) / npass;
    uint64_t *kin = keys_a, *kout = keys_b;
    uint32_t *vin = vals_a, *vout = vals_b;
    bool in_b = false;
    for (int shift = lo; shift < hi; shift += per) {
        const int bits = min(per, hi - shift);
        const unsigned mask = (1u << bits) - 1u;
        cudaError_t e;
        if (nd)
            e = bits > 9 ? rs_pass<1024, true>(kin, kout, vin, vout, n, nd, shift, mask, g, counts,
                                               totals, status, st)
                         : rs_pass<512, true>(kin, kout, vin, vout, n, nd, shift, mask, g, counts,
                                              totals, status, st);
        else
            e = bits > 9 ? rs_pass<1024, false>(kin, kout, vin, vout, n, nd, shift, mask, g,
                                                counts, totals, status, st)
                         : rs_pass<512, false>(kin, kout, vin, vout, n, nd, shift, mask, g, counts,
                                               totals, status, st);
        if (e != cudaSuccess) return e;
        uint64_t *tk = kin;
        kin = kout;
        kout = tk;
        uint32_t *tv = vin;
        vin = vout;
        vout = tv;
        in_b = !in_b;
    }
    *result_in_b = in_b;
    return cudaGetLastError();
}

size_t scan_temp_bytes(long long n) {
    long long nb = (n + SC_CHUNK - 1) / SC_CHUNK;
    return (size_t)(nb + 1) * 8 + 256;
}

cudaError_t scan_u32_to_u64(const uint32_t *in, unsigned long long *out, long long n, void *tmp,
                            cudaStream_t st) {
    return scan_impl<uint32_t, unsigned long long>(in, out, n, tmp, st);
}

cudaError_t scan_u32_to_u32(const uint32_t *in, uint32_t *out, long long n, void *tmp,
                            cudaStream_t st) {
    return scan_impl<uint32_t, uint32_t>(in, out, n, tmp, st);
}

size_t hsp_sort_temp_bytes(long long n) {
    n = n > 0 ? n : 1;
    return (size_t)n * (8 + 8 + 4 + 4 + sizeof(Hsp)) + radix_sort_temp_bytes(n) + 1024;
}

cudaError_t hsp_sort(Hsp *hsps, long long n, int tbits, int qbits, void *tmp, uint32_t *status,
                     cudaStream_t st) {
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
    Hsp *hb = reinterpret_cast<Hsp *>(take((size_t)n * sizeof(Hsp)));
    void *rt = take(radix_sort_temp_bytes(n));
    g_launches++;
    hsp_keys<<<grid_for(n), BLOCK, 0, st>>>(hsps, n, qbits, ka, va);
    bool in_b = false;
    // strand sits at bit 62; tpos and qpos below it
    cudaError_t e = radix_sort(ka, kb, va, vb, n, 0, qbits + tbits, rt, &in_b, status, st);
    if (e != cudaSuccess) return e;
    uint64_t *k1 = in_b ? kb : ka, *k2 = in_b ? ka : kb;
    unsigned *v1 = in_b ? vb : va, *v2 = in_b ? va : vb;
    e = radix_sort(k1, k2, v1, v2, n, 62, 63, rt, &in_b, status, st);
    if (e != cudaSuccess) return e;
    uint64_t *kf = in_b ? k2 : k1;
    unsigned *vf = in_b ? v2 : v1;
    g_launches += 2;
    hsp_gather<<<grid_for(n), BLOCK, 0, st>>>(hsps, vf, n, hb);
    hsp_fix_runs<<<grid_for(n), BLOCK, 0, st>>>(hb, kf, n);
    cudaMemcpyAsync(hsps, hb, (size_t)n * sizeof(Hsp), cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError();
}

}  // namespace sfe
