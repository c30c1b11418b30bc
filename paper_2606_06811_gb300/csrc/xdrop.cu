// Per-diagonal skip and ungapped X-drop (Algorithm 1 with X-drop as the
// extension; the X-drop filter of Section 2 and Section 8).
//
// The hits of one query tile arrive sorted by (diagonal, t). Each diagonal is a
// segment, and its loop-carried dependency (skip a hit with t < E, where E is
// the end of the last extended HSP on that diagonal) is resolved exactly by
// walking the segment in order. Diagonals are independent, so they are walked
// in parallel, in two tiers:
//
//  * lane tier: one thread walks one diagonal. Most hits are random and their
//    extensions stop within a few dozen bases, so a thread scores one base per
//    step (2-bit bases from 16-base register windows, scores from a 16-entry
//    shared-memory table) with no inter-thread traffic. When a side passes
//    `lane_cap` bases, the thread stops and queues (segment, hit, E): its warp
//    would otherwise wait on one long extension.
//  * warp tier: one warp resumes each queued diagonal and finishes it with
//    32-base chunks, as the warp-per-hit design that the paper credits to
//    SegAlign (Section 2, Section 8): lane i scores base i, a __shfl_up scan
//    gives the running sum and its running maximum, __ballot finds the first
//    base with max - sum > X, and the earliest maximum gives the HSP end.
//
// Both tiers compute exactly the serial definition: same bases scored, same
// HSP, same E, same cells.
#include <climits>

#include "sfe_internal.cuh"

namespace sfe {

namespace {

constexpr int W_BLOCK = 256;
constexpr int SCORE_LIMIT = 1 << 30;  // a best score above this flags overflow

__global__ void seg_flags_kernel(const uint64_t *__restrict__ hits, long long n,
                                 uint32_t *__restrict__ flags) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    flags[i] = (i == 0) || ((hits[i] >> 32) != (hits[i - 1] >> 32));
}

__global__ void seg_write_kernel(const uint32_t *__restrict__ flags,
                                 const unsigned long long *__restrict__ scan, long long n,
                                 uint32_t *__restrict__ seg_start) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n && flags[i]) seg_start[scan[i]] = (uint32_t)i;
    if (i == n) seg_start[scan[n]] = (uint32_t)n;
}

struct Side {
    int best;    // maximum of the running sum (0 for the empty extension)
    int blen;    // earliest length at which `best` is reached
    int scored;  // bases scored
};

// Lane tier, right side: bases pt+n, pq+n for n = 0 .. avail-1.
// Returns false when `cap` bases were scored without a stop (hand-off).
__device__ __forceinline__ bool lane_right(const uint32_t *__restrict__ T,
                                           const uint32_t *__restrict__ Q, long long pt,
                                           long long pq, int avail, int X, int cap,
                                           const int *lut, Side &r, uint32_t &status) {
    int sum = 0, best = 0, blen = 0, n = 0;
    while (n < avail) {
        if (n >= cap) return false;
        uint32_t tw = win16(T, pt + n), qw = win16(Q, pq + n);
        int m = min(16, avail - n);
        int stop = -1;
#pragma unroll
        for (int j = 0; j < 16; j++) {
            if (j >= m) break;
            int s = lut[((tw >> (2 * j)) & 3u) * 4u + ((qw >> (2 * j)) & 3u)];
            sum += s;
            if (sum > best) {
                best = sum;
                blen = n + j + 1;
            }
            if (best - sum > X) {
                stop = j;
                break;
            }
        }
        if (best > SCORE_LIMIT) status |= ST_SCORE_OVERFLOW;
        if (stop >= 0) {
            n += stop + 1;
            r = {best, blen, n};
            return true;
        }
        n += m;
    }
    r = {best, blen, n};
    return true;
}

// Lane tier, left side: bases pt-1-n, pq-1-n for n = 0 .. avail-1.
__device__ __forceinline__ bool lane_left(const uint32_t *__restrict__ T,
                                          const uint32_t *__restrict__ Q, long long pt,
                                          long long pq, int avail, int X, int cap,
                                          const int *lut, Side &r, uint32_t &status) {
    int sum = 0, best = 0, blen = 0, n = 0;
    while (n < avail) {
        if (n >= cap) return false;
        // bases [p-15, p] with p = pt-1-n: base p sits in bits 30-31
        uint32_t tw = win16(T, pt - 16 - n), qw = win16(Q, pq - 16 - n);
        int m = min(16, avail - n);
        int stop = -1;
#pragma unroll
        for (int j = 0; j < 16; j++) {
            if (j >= m) break;
            int s = lut[((tw >> (30 - 2 * j)) & 3u) * 4u + ((qw >> (30 - 2 * j)) & 3u)];
            sum += s;
            if (sum > best) {
                best = sum;
                blen = n + j + 1;
            }
            if (best - sum > X) {
                stop = j;
                break;
            }
        }
        if (best > SCORE_LIMIT) status |= ST_SCORE_OVERFLOW;
        if (stop >= 0) {
            n += stop + 1;
            r = {best, blen, n};
            return true;
        }
        n += m;
    }
    r = {best, blen, n};
    return true;
}

__device__ __forceinline__ int lane_span(const uint32_t *__restrict__ T,
                                         const uint32_t *__restrict__ Q, long long t, long long q,
                                         int span, const int *lut) {
    uint64_t tv = (uint64_t)win16(T, t) | ((uint64_t)win16(T, t + 16) << 32);
    uint64_t qv = (uint64_t)win16(Q, q) | ((uint64_t)win16(Q, q + 16) << 32);
    int s = 0;
    for (int k = 0; k < span; k++)
        s += lut[((tv >> (2 * k)) & 3u) * 4u + ((qv >> (2 * k)) & 3u)];
    return s;
}

__device__ __forceinline__ void emit(const WalkParams &wp, long long t, long long q, int lblen,
                                     int rblen, long long score, uint32_t &status) {
    unsigned long long idx = atomicAdd(&wp.ctr->hsps, 1ull);
    if (idx < wp.hsp_cap) {
        Hsp h;
        h.strand = wp.strand;
        h.tpos = (int32_t)(t - lblen);
        h.qpos = (int32_t)(q - lblen);
        h.len = wp.span + lblen + rblen;
        h.score = (int32_t)score;
        wp.hsps[idx] = h;
    } else {
        status |= ST_HSP_OVERFLOW;
    }
}

__global__ void __launch_bounds__(W_BLOCK) walk_lanes_kernel(
    const uint64_t *__restrict__ hits, const uint32_t *__restrict__ seg_start,
    const unsigned long long *__restrict__ nseg_ptr, WalkParams wp) {
    __shared__ int lut[16];
    if (threadIdx.x < 16) lut[threadIdx.x] = wp.scores[threadIdx.x];
    __syncthreads();
    const unsigned long long nseg = *nseg_ptr;
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned long long ext = 0, cells = 0, tasks = 0;
    uint32_t status = 0;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < (long long)nseg;
         s += stride) {
        tasks++;
        uint32_t i = seg_start[s], end = seg_start[s + 1];
        const long long D = (long long)((hits[i] >> 32) & 0x7FFFFFFFu);
        int E = wp.Ecarry ? wp.Ecarry[D] : INT_MIN;
        bool handed = false;
        int cap = wp.lane_cap;
        while (i < end) {
            const long long t = (long long)(uint32_t)hits[i];
            if (t < E) {
                i++;
                continue;
            }
            const long long q = t - D + wp.qoff;
            const long long pt = t + wp.span, pq = q + wp.span;
            Side r, l;
            int ravail = (int)min(wp.tlen - pt, wp.qlen - pq);
            int lavail = (int)min(t, q);
            bool ok = lane_right(wp.T, wp.Q, pt, pq, ravail, wp.xdrop, cap, lut, r, status) &&
                      lane_left(wp.T, wp.Q, t, q, lavail, wp.xdrop, cap, lut, l, status);
            if (!ok) {
                unsigned int slot = atomicAdd(wp.queue_len, 1u);
                if (slot < wp.queue_cap) {
                    wp.queue[slot] = make_uint4((uint32_t)s, i, (uint32_t)E, 0u);
                    handed = true;
                    break;
                }
                // queue full: this lane finishes the diagonal itself
                cap = INT_MAX;
                continue;
            }
            const int s0 = lane_span(wp.T, wp.Q, t, q, wp.span, lut);
            const long long score = (long long)s0 + r.best + l.best;
            if (score > INT_MAX) status |= ST_SCORE_OVERFLOW;
            ext++;
            cells += (unsigned long long)(wp.span + r.scored + l.scored);
            const bool pass = score >= wp.thresh;
            if (pass) emit(wp, t, q, l.blen, r.blen, score, status);
            if (pass || !(wp.flags & SFE_SKIP_PASSING_ONLY)) E = (int)(t + wp.span + r.blen);
            i++;
        }
        if (!handed && wp.Ecarry) wp.Ecarry[D] = E;
    }
    // one atomic per warp for each counter
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ext += __shfl_down_sync(0xffffffffu, ext, o);
        cells += __shfl_down_sync(0xffffffffu, cells, o);
        tasks += __shfl_down_sync(0xffffffffu, tasks, o);
        status |= __shfl_down_sync(0xffffffffu, status, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (ext) atomicAdd(&wp.ctr->extended, ext);
        if (cells) atomicAdd(&wp.ctr->cells, cells);
        if (tasks) atomicAdd(&wp.ctr->lane_tasks, tasks);
        if (status) atomicOr(&wp.ctr->status, status);
    }
}

// ------------------------------------------------------------------ warps

__device__ __forceinline__ int warp_incl_sum(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

__device__ __forceinline__ int warp_incl_max(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v = max(v, y);
    }
    return v;
}

// One side in 32-base chunks; dir = +1 (right: bases p0 + k) or -1 (left:
// bases p0 - k). All lanes return the same result.
__device__ __forceinline__ Side warp_side(const uint32_t *__restrict__ T,
                                          const uint32_t *__restrict__ Q, long long pt0,
                                          long long pq0, int dir, int avail, int X,
                                          const int *lut, int lane, uint32_t &status) {
    int carry = 0, best = 0, blen = 0, scored = avail;
    for (int k0 = 0; k0 < avail; k0 += 32) {
        const int k = k0 + lane;
        const bool valid = k < avail;
        int s = 0;
        if (valid) {
            uint32_t tb = base_at(T, pt0 + dir * (long long)k);
            uint32_t qb = base_at(Q, pq0 + dir * (long long)k);
            s = lut[tb * 4u + qb];
        }
        const int P = warp_incl_sum(s, lane) + carry;
        const int Mx = max(warp_incl_max(P, lane), best);
        const unsigned stopm = __ballot_sync(0xffffffffu, valid && (Mx - P > X));
        const int nvalid = min(32, avail - k0);
        const int last = stopm ? __ffs(stopm) - 1 : nvalid - 1;
        const int bl = __shfl_sync(0xffffffffu, Mx, last);
        if (bl > best) {
            const unsigned m = __ballot_sync(0xffffffffu, lane <= last && P == bl);
            blen = k0 + __ffs(m);
            best = bl;
        }
        if (best > SCORE_LIMIT) status |= ST_SCORE_OVERFLOW;
        if (stopm) {
            scored = k0 + last + 1;
            break;
        }
        carry = __shfl_sync(0xffffffffu, P, 31);
    }
    return {best, blen, scored};
}

__global__ void __launch_bounds__(W_BLOCK) walk_warps_kernel(const uint64_t *__restrict__ hits,
                                                             const uint32_t *__restrict__ seg_start,
                                                             WalkParams wp) {
    __shared__ int lut[16];
    if (threadIdx.x < 16) lut[threadIdx.x] = wp.scores[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const unsigned long long nq = min((unsigned long long)*wp.queue_len, wp.queue_cap);
    unsigned long long ext = 0, cells = 0, tasks = 0;
    uint32_t status = 0;
    for (long long e = warp; e < (long long)nq; e += nwarps) {
        const uint4 it = wp.queue[e];
        tasks++;
        uint32_t i = it.y;
        const uint32_t end = seg_start[it.x + 1];
        int E = (int)it.z;
        const long long D = (long long)((hits[i] >> 32) & 0x7FFFFFFFu);
        while (i < end) {
            const long long t = (long long)(uint32_t)hits[i];
            if (t < E) {
                i++;
                continue;
            }
            const long long q = t - D + wp.qoff;
            // seed span: lanes 0..span-1
            int s = 0;
            if (lane < wp.span) s = lut[base_at(wp.T, t + lane) * 4u + base_at(wp.Q, q + lane)];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            const long long pt = t + wp.span, pq = q + wp.span;
            const int ravail = (int)min(wp.tlen - pt, wp.qlen - pq);
            const int lavail = (int)min(t, q);
            const Side r = warp_side(wp.T, wp.Q, pt, pq, +1, ravail, wp.xdrop, lut, lane, status);
            const Side l = warp_side(wp.T, wp.Q, t - 1, q - 1, -1, lavail, wp.xdrop, lut, lane,
                                     status);
            const long long score = (long long)s + r.best + l.best;
            if (score > INT_MAX) status |= ST_SCORE_OVERFLOW;
            ext++;
            cells += (unsigned long long)(wp.span + r.scored + l.scored);
            const bool pass = score >= wp.thresh;
            if (pass && lane == 0) emit(wp, t, q, l.blen, r.blen, score, status);
            if (pass || !(wp.flags & SFE_SKIP_PASSING_ONLY)) E = (int)(t + wp.span + r.blen);
            i++;
        }
        if (wp.Ecarry && lane == 0) wp.Ecarry[D] = E;
    }
    if (lane == 0) {
        if (ext) atomicAdd(&wp.ctr->extended, ext);
        if (cells) atomicAdd(&wp.ctr->cells, cells);
        if (tasks) atomicAdd(&wp.ctr->warp_tasks, tasks);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) status |= __shfl_down_sync(0xffffffffu, status, o);
    if (lane == 0 && status) atomicOr(&wp.ctr->status, status);
}

inline unsigned grid_for(long long n, int block = BLOCK) {
    return (unsigned)((n + block - 1) / block);
}

int g_sms = 0;
int sms() {
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    return g_sms;
}

}  // namespace

size_t segments_temp_bytes(long long n) { return scan_temp_bytes(n); }

cudaError_t launch_segments(const uint64_t *hits, long long n, uint32_t *flags,
                            unsigned long long *scan, uint32_t *seg_start, void *tmp,
                            cudaStream_t st) {
    if (n > 0) seg_flags_kernel<<<grid_for(n), BLOCK, 0, st>>>(hits, n, flags);
    cudaError_t e = scan_u32_to_u64(flags, scan, n, tmp, st);
    if (e != cudaSuccess) return e;
    seg_write_kernel<<<grid_for(n + 1), BLOCK, 0, st>>>(flags, scan, n, seg_start);
    return cudaGetLastError();
}

cudaError_t launch_walk_lanes(const uint64_t *hits, const uint32_t *seg_start,
                              const unsigned long long *nseg_dev, long long nseg_max,
                              WalkParams wp, cudaStream_t st) {
    if (nseg_max <= 0) return cudaSuccess;
    long long want = grid_for(nseg_max, W_BLOCK);
    long long cap = 16LL * sms();
    unsigned grid = (unsigned)(want < cap ? want : cap);
    walk_lanes_kernel<<<grid, W_BLOCK, 0, st>>>(hits, seg_start, nseg_dev, wp);
    return cudaGetLastError();
}

cudaError_t launch_walk_warps(const uint64_t *hits, const uint32_t *seg_start, WalkParams wp,
                              int grid_warps, cudaStream_t st) {
    if (grid_warps <= 0) grid_warps = 8 * sms() * (W_BLOCK / 32);
    unsigned grid = (unsigned)((grid_warps * 32 + W_BLOCK - 1) / W_BLOCK);
    walk_warps_kernel<<<grid, W_BLOCK, 0, st>>>(hits, seg_start, wp);
    return cudaGetLastError();
}

}  // namespace sfe
