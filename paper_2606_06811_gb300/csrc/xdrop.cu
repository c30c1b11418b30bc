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

struct Side {
    int best;    // maximum of the running sum (0 for the empty extension)
    int blen;    // earliest length at which `best` is reached
    int scored;  // bases scored
};

// Where one diagonal's hits live: its pair's sequences and lengths, and its
// strand. For a single pair everything comes from the launch parameters.
struct SegCtx {
    const uint32_t *Q;  // packed query strand buffer
    long long tb, qb;   // global base of the pair's target and query strand
    long long tlen, qlen, qoff;
    long long D;        // local diagonal index
    int strand, pair;
};

template <bool BATCH>
__device__ __forceinline__ void seg_ctx(const WalkParams &wp, uint32_t word, SegCtx &c) {
    if (BATCH) {
        c.pair = (int)(word >> (wp.dbits + 1));
        c.strand = (int)((word >> wp.dbits) & 1u);
        c.D = (long long)(word & ((1u << wp.dbits) - 1u));
        const PairInfo P = wp.pairs[c.pair];
        c.tb = P.toff;
        c.qb = c.strand ? P.qoff_rc : P.qoff;
        c.tlen = P.tlen;
        c.qlen = P.qlen;
        c.Q = c.strand ? wp.Qrc : wp.Q;
    } else {
        c.pair = 0;
        c.strand = wp.strand;
        c.D = (long long)(word & 0x7FFFFFFFu);
        c.tb = 0;
        c.qb = 0;
        c.tlen = wp.tlen;
        c.qlen = wp.qlen;
        c.Q = wp.Q;
    }
    c.qoff = c.qlen - wp.span;
}

__device__ __forceinline__ void log_ext(const WalkParams &wp, const SegCtx &c, long long t,
                                        long long q, int right, int left) {
    if (!wp.elog || !ext_sampled(wp.elog_every, c.pair, c.strand, t, q)) return;
    const unsigned long long idx = atomicAdd(&wp.ctr->ext_logged, 1ull);
    if (idx < wp.elog_cap) {
        sfe_ext_record r;
        r.pair = c.pair;
        r.strand = c.strand;
        r.t = (int32_t)t;
        r.q = (int32_t)q;
        r.right = right;
        r.left = left;
        wp.elog[idx] = r;
    }
}

template <bool BATCH>
__device__ __forceinline__ void emit(const WalkParams &wp, const SegCtx &c, long long t,
                                     long long q, int lblen, int rblen, long long score,
                                     uint32_t &status) {
    unsigned long long idx = atomicAdd(&wp.ctr->hsps, 1ull);
    if (idx < wp.hsp_cap) {
        if (BATCH) {
            BatchHsp h;
            h.pair = c.pair;
            h.strand = c.strand;
            h.tpos = (int32_t)(t - lblen);
            h.qpos = (int32_t)(q - lblen);
            h.len = wp.span + lblen + rblen;
            h.score = (int32_t)score;
            wp.bhsps[idx] = h;
        } else {
            Hsp h;
            h.strand = c.strand;
            h.tpos = (int32_t)(t - lblen);
            h.qpos = (int32_t)(q - lblen);
            h.len = wp.span + lblen + rblen;
            h.score = (int32_t)score;
            wp.hsps[idx] = h;
        }
    } else {
        status |= ST_HSP_OVERFLOW;
    }
}

// 2-bit groups of x in reverse order (group i -> group 15 - i).
__device__ __forceinline__ uint32_t rev2(uint32_t x) {
    x = __brev(x);
    return ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);
}

__device__ __forceinline__ uint32_t diag_of(uint64_t h) { return (uint32_t)(h >> 32); }

// First index j > i whose diagonal word differs from `d`, the word of hits[i]
// (hits are sorted by diagonal word). Diagonals are short, so the search
// gallops from i (i + 1, i + 2, i + 4, ...: a few nearby loads) before it
// bisects, instead of bisecting the whole array.
__device__ __forceinline__ uint32_t segment_end(const uint64_t *__restrict__ hits, uint32_t i,
                                                uint32_t n, uint32_t d) {
    uint32_t lo = i, hi, step = 1;  // diag(hits[lo]) <= d
    while (true) {
        hi = (n - lo > step) ? lo + step : n;
        if (hi >= n || diag_of(hits[hi]) > d) break;
        lo = hi;
        step <<= 1;
    }
    uint32_t a = lo + 1, b = hi;  // the first index in (lo, hi] with a larger word
    while (a < b) {
        const uint32_t mid = a + (b - a) / 2;
        if (diag_of(hits[mid]) <= d)
            a = mid + 1;
        else
            b = mid;
    }
    return a;
}

// Score of the seed span [t, t + span) from a table of pair sums: entry
// (ta | tb << 2 | qa << 4 | qb << 6) = M[ta][qa] + M[tb][qb].
__device__ __forceinline__ int span_score(const uint32_t *__restrict__ T,
                                          const uint32_t *__restrict__ Q, long long t, long long q,
                                          int span, const int *psum, const int *lut) {
    const uint64_t tv = (uint64_t)win16(T, t) | ((uint64_t)win16(T, t + 16) << 32);
    const uint64_t qv = (uint64_t)win16(Q, q) | ((uint64_t)win16(Q, q + 16) << 32);
    int s = 0;
    const int pairs = span >> 1;
    for (int m = 0; m < pairs; m++)
        s += psum[((uint32_t)(tv >> (4 * m)) & 15u) | (((uint32_t)(qv >> (4 * m)) & 15u) << 4)];
    if (span & 1) {
        const int k = span - 1;
        s += lut[((uint32_t)(tv >> (2 * k)) & 3u) * 4u + ((uint32_t)(qv >> (2 * k)) & 3u)];
    }
    return s;
}

// State of one extension side in the lane tier: the running maximum, the
// running sum's drop below it (d = best - sum >= 0), the earliest length that
// reached the maximum and the bases scored.
struct LaneSide {
    int n;     // bases scored
    int d;     // best - running sum
    int best;  // running maximum (0 for the empty extension)
    int blen;  // earliest length reaching `best`
    bool done;
};

// The 2-bit codes in bits 0..15 of x, one per nibble (code k -> bits 4k, 4k + 1).
__device__ __forceinline__ uint32_t spread8(uint32_t x, uint32_t sel) {
    x = __byte_perm(x, 0u, sel);  // two bytes of x into the low bytes of the halfwords
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    return (x | (x << 2)) & 0x33333333u;
}

// Cell planes: a sequence at 4 bits per base, nibble k of word w holding the
// code of base 8w + k, target codes in bits 2-3 of their nibble and query
// codes in bits 0-1, so the OR of a target and a query window is the packed
// window's table index per cell with no bit shuffling. Sixteen nibbles from
// base p (p >= -16): three word loads and two funnel shifts. A plane has
// PLANE_PAD zero words before base 0 and after its last word. A left window
// reads the 16 bases that end where the side stands and takes their nibbles
// in reverse order (a constant index per cell), so both sides of a hit read
// the same lines of the plane.
__device__ __forceinline__ uint2 plane_win16(const uint32_t *__restrict__ P, int p) {
    const int w = p >> 3;
    const uint32_t sh = (uint32_t)(p & 7) * 4u;
    const uint32_t a = __ldg(P + w), b = __ldg(P + w + 1), c = __ldg(P + w + 2);
    return make_uint2(__funnelshift_r(a, b, sh), __funnelshift_r(b, c, sh));
}

// Largest X for which the packed-key window below cannot overflow int32
// (scores are limited to |M| <= 2^20).
constexpr int PACKED_X_LIMIT = 1 << 23;

// Scores the next 16 bases of a side whose next base is (pt, pq) going `dir`
// (+1 forward, -1 backward; a backward window is read bit-reversed).
//
// The window works on sums relative to the current maximum, so its values stay
// within X + 16 max|score| whatever the side's length. With PACKED, the table
// lut64 holds 64 * M - 1, and one accumulator carries both the running sum and
// the count of scored cells: acc = 64 * sum - cells. Since cells <= 16 < 64, a
// larger acc is a larger sum, or the same sum reached after fewer cells, so
// max(acc) tracks the maximum and its earliest position at once (the previous
// maximum is key 0 and wins ties). best - sum > X exactly when
// max(acc) - acc >= 64 * (X + 1), that is when acc + 64 * (X + 1) > max(acc)
// fails. A predicate `on` freezes acc once the side stops. Per cell: one
// table load, an add under the predicate, a max and a compare folded into the
// predicate (measured 0.7% faster than multiplying the score by a 0/1 flag).
//
// PLANES (packed, one pair): the window comes from the cell planes of
// `wp` instead of the 2-bit words; cell j of a left window is nibble 15 - j.
template <bool PACKED, bool PLANES = false, bool LOCAL = false>
__device__ __forceinline__ void lane_window(const uint32_t *__restrict__ T,
                                            const uint32_t *__restrict__ Q, long long pt,
                                            long long pq, int dir, int avail, int X,
                                            const int *lut, const int *lut64, LaneSide &sd,
                                            const WalkParams &wp) {
    uint32_t tw = 0, qw = 0;
    uint2 zp = make_uint2(0u, 0u);
    if (PLANES) {
        // one pair: positions are local and below 2^31
        const int pt32 = (int)pt, pq32 = (int)pq;
        const uint2 tz = plane_win16(wp.TN, dir > 0 ? pt32 + sd.n : pt32 - sd.n - 16);
        const uint2 qz = plane_win16(wp.QN, dir > 0 ? pq32 + sd.n : pq32 - sd.n - 16);
        zp = make_uint2(tz.x | qz.x, tz.y | qz.y);
    } else {
        if (LOCAL) {  // one pair: positions below 2^31
            const int wt = dir > 0 ? (int)pt + sd.n : (int)pt - sd.n - 16;
            const int wq = dir > 0 ? (int)pq + sd.n : (int)pq - sd.n - 16;
            tw = __funnelshift_r(__ldg(T + (wt >> 4)), __ldg(T + (wt >> 4) + 1),
                                 (uint32_t)(wt & 15) * 2u);
            qw = __funnelshift_r(__ldg(Q + (wq >> 4)), __ldg(Q + (wq >> 4) + 1),
                                 (uint32_t)(wq & 15) * 2u);
        } else {
            const long long wt = dir > 0 ? pt + sd.n : pt - sd.n - 16;
            const long long wq = dir > 0 ? pq + sd.n : pq - sd.n - 16;
            tw = win16(T, wt);
            qw = win16(Q, wq);
        }
        if (dir < 0) {
            tw = rev2(tw);
            qw = rev2(qw);
        }
    }
    const int lim = avail - sd.n;
    int cnt = 0, a = 1, bj = -1, gain = 0, sum = 0;
    if (PACKED) {
        const int thr = 64 * (X + 1);
        int acc = -64 * sd.d;
        int bk = 0;  // key of the current maximum
        // table index of cell j (4 * t + q) in nibble j of z[j / 8]
        const uint32_t z[2] = {
            PLANES ? zp.x : spread8(tw, 0x4140u) * 4u + spread8(qw, 0x4140u),
            PLANES ? zp.y : spread8(tw, 0x4342u) * 4u + spread8(qw, 0x4342u)};
        if (lim >= 16) {
            bool on = true;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int k = (PLANES && dir < 0) ? 15 - j : j;  // nibble of cell j
                const int sc = lut64[(z[k >> 3] >> (4 * (k & 7))) & 15u];
                acc = on ? acc + sc : acc;
                bk = max(bk, acc);
                on = on && (acc + thr > bk);
            }
            a = on;
        } else {
            bool on = true;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int k = (PLANES && dir < 0) ? 15 - j : j;
                const int sc = lut64[(z[k >> 3] >> (4 * (k & 7))) & 15u];
                on = on && j < lim;
                acc = on ? acc + sc : acc;
                bk = max(bk, acc);
                on = on && (acc + thr > bk);
            }
            a = on;
        }
        cnt = (-acc) & 63;
        sum = (acc + cnt) >> 6;
        if (bk > 0) {
            gain = (bk + 63) >> 6;
            bj = 64 * gain - bk - 1;
        }
    } else {
        sum = -sd.d;
        int lbest = 0;
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const int sc = lut[((tw >> (2 * j)) & 3u) * 4u + ((qw >> (2 * j)) & 3u)];
            a = j < lim ? a : 0;
            sum = sc * a + sum;
            cnt += a;
            const bool nb = sum > lbest;
            lbest = nb ? sum : lbest;
            bj = nb ? j : bj;
            a = (lbest - sum <= X) ? a : 0;
        }
        gain = lbest;
    }
    if (bj >= 0) {
        sd.blen = sd.n + bj + 1;
        sd.best += gain;
    }
    sd.d = gain - sum;
    sd.n += cnt;
    sd.done = a == 0 || sd.n >= avail;
}

template <bool BATCH>
__device__ void warp_walk_diagonal(const uint64_t *__restrict__ hits, uint32_t nhits, uint32_t i,
                                   int E, const WalkParams &wp, const int *lut, int lane,
                                   unsigned long long &ext, unsigned long long &cells,
                                   uint32_t &status);

// The warp tier of the persistent walk: a warp whose lanes are out of lane
// work takes hand-off entries in order and finishes each entry's diagonal.
// An entry whose producer has not published it in time (its CTA may not be
// resident yet while this one waits) is left, with the rest of the queue, to
// the follow-up warp launch on the same stream, which runs after every
// producer has finished.
template <bool BATCH>
__device__ __forceinline__ void drain_queue(const uint64_t *__restrict__ hits, uint32_t n,
                                            const WalkParams &wp, const int *lut, int lane,
                                            uint32_t &status) {
    // this warp's lanes are out of work: consume the hand-off queue
    __threadfence();
    if (lane == 0) atomicAdd(wp.warps_done, 1u);
    const unsigned total_warps = gridDim.x * (W_BLOCK / 32);
    unsigned long long wext = 0, wcells = 0, wtasks = 0, wdeferred = 0;
    while (true) {
        unsigned e = 0;
        if (lane == 0) e = atomicAdd(wp.queue_take, 1u);
        e = __shfl_sync(0xffffffffu, e, 0);
        if (e >= wp.queue_cap) break;
        int state = 0;  // 1: entry ready, 2: no entry will come, 3: waited too long
        long long spins = 0;
        unsigned backoff = 32;  // ns: a waiting warp leaves the issue slots to working ones
        while (state == 0) {
            if (lane == 0) {
                volatile uint4 *qe = wp.queue + e;
                if (qe->z == wp.epoch) {
                    state = 1;
                } else {
                    const unsigned wd = *(volatile unsigned *)wp.warps_done;
                    const unsigned ql = *(volatile unsigned *)wp.queue_len;
                    if (wd >= total_warps && e >= min(ql, (unsigned)wp.queue_cap)) state = 2;
                    else if (++spins > wp.spin_limit) state = 3;
                    else {
                        __nanosleep(backoff);
                        backoff = min(backoff * 2u, 1024u);
                    }
                }
            }
            state = __shfl_sync(0xffffffffu, state, 0);
        }
        if (state == 3) wdeferred++;
        if (state != 1) break;
        __threadfence();
        volatile uint4 *qe = wp.queue + e;
        const uint32_t hi_idx = qe->x;
        const int hi_E = (int)qe->y;
        wtasks++;
        warp_walk_diagonal<BATCH>(hits, n, hi_idx, hi_E, wp, lut, lane, wext, wcells, status);
        if (lane == 0) qe->w = wp.epoch;  // done: the follow-up launch skips it
    }
    if (lane == 0) {
        if (wext) atomicAdd(&wp.ctr->extended, wext);
        if (wcells) {
            atomicAdd(&wp.ctr->cells, wcells);
            atomicAdd(&wp.ctr->warp_cells, wcells);
        }
        if (wtasks) atomicAdd(&wp.ctr->warp_tasks, wtasks);
        if (wdeferred) atomicAdd(&wp.ctr->deferred, wdeferred);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) status |= __shfl_down_sync(0xffffffffu, status, o);
}

// Lane tier. Lane k owns the diagonals that start in hit range
// [k*chunk, (k+1)*chunk) and streams through its hits in order, with the next
// hit prefetched. The lanes of a warp advance in lock step, one iteration at
// a time: (1) each lane without a hit in progress looks at its next hit
// (closing its diagonal and opening the next when the diagonal word changes)
// and skips it if t < E, or starts extending it; (2) every lane whose
// right side is still open scores its next 16 bases; (3) the same for the left
// sides; (4) lanes whose two sides are closed advance E and, when the two
// extensions could reach the threshold with any seed span, score the span
// from a pair-sum table and emit the HSP if it passes. Most
// hits finish in one iteration, so the warp stays converged while its lanes
// work on different hits and diagonals. A side that passes `lane_cap` bases
// hands the rest of its diagonal to the warp tier.
template <bool PACKED, bool BATCH, bool PERSIST, bool PLANES = false>
__global__ void __launch_bounds__(W_BLOCK, PERSIST ? 1 : 0) walk_lanes_kernel(const uint64_t *__restrict__ hits,
                                                             uint32_t n, uint32_t chunk,
                                                             WalkParams wp) {
    __shared__ int lut[16];
    __shared__ int lut64[16];
    __shared__ int psum[256];
    if (threadIdx.x < 16) {
        lut[threadIdx.x] = wp.scores[threadIdx.x];
        lut64[threadIdx.x] = 64 * wp.scores[threadIdx.x] - 1;
    }
    {
        const int e = threadIdx.x;  // W_BLOCK == 256 entries
        psum[e] = wp.scores[(e & 3) * 4 + ((e >> 4) & 3)] +
                  wp.scores[((e >> 2) & 3) * 4 + ((e >> 6) & 3)];
    }
    __syncthreads();
    const int span = wp.span, X = wp.xdrop;
    if (PERSIST && wp.phantom && blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd(wp.queue_len, 1u);  // test hook: a queue slot nobody will publish
    uint32_t nchunks = wp.nchunks;
    if (wp.nd) {  // the hit count lives on the device: ranges and chunks follow it
        n = (uint32_t)min((unsigned long long)n, *wp.nd);
        if (PERSIST)
            nchunks = (n + wp.chunk - 1) / wp.chunk;
        else
            chunk = max(16u, (uint32_t)((n + (unsigned long long)gridDim.x * blockDim.x - 1) /
                                        ((unsigned long long)gridDim.x * blockDim.x)));
    }
    // upper bound of a seed span's score: the span is scored only for hits
    // whose extensions could lift the HSP to the threshold
    int maxsc = lut[0];
#pragma unroll
    for (int k = 1; k < 16; k++) maxsc = max(maxsc, lut[k]);
    const long long s0_bound = (long long)span * maxsc;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long lo64 = PERSIST ? 0 : tid * (long long)chunk;
    uint32_t range_end = PERSIST ? 0u : (uint32_t)min((long long)n, lo64 + chunk);

    uint32_t i = (uint32_t)min((long long)n, lo64);
    // a diagonal that started before this range belongs to the previous lane
    if (!PERSIST && i > 0 && i < range_end && diag_of(hits[i]) == diag_of(hits[i - 1]))
        i = segment_end(hits, i, n, diag_of(hits[i]));
    uint64_t cur = (!PERSIST && i < n) ? hits[i] : ~0ull, nxt = ~0ull;
    bool in_seg = false, handed = false, busy = false, done = !PERSIST && i >= range_end;
    uint32_t D = 0;
    SegCtx c;
    seg_ctx<BATCH>(wp, 0u, c);
    // positions in 32 bits (sequences are shorter than 2^31 bases); per
    // diagonal: q = t + dq, and the room left on each side. (With 64-bit
    // positions and window addresses the walk took 9.98 ms per step on the
    // 10 Mb pair against 9.54; 9.96 against 9.66 with the 2-bit windows.)
    int t = 0, q = 0, dq = 0, tr = 0, qr = 0;
    int E = INT_MIN, cap = wp.lane_cap, ravail = 0, lavail = 0;
    LaneSide R{0, 0, 0, 0, true}, L{0, 0, 0, 0, true};
    unsigned long long ext = 0, cells = 0, tasks = 0, shadow = 0;
    uint32_t status = 0;

    while (true) {
        // (1) fetch: a lane without a hit in progress looks at one hit per
        // iteration (straight-line, so the lanes stay converged)
        if (!busy && !done) {
            if (!in_seg || i >= n || diag_of(cur) != D) {
                // diagonal boundary: close the current one, open the next
                if (in_seg && !handed && wp.Ecarry) wp.Ecarry[D & 0x7FFFFFFFu] = E;
                in_seg = false;
                if (i >= range_end) {
                    if (PERSIST) {
                        // take the next chunk of hits from the work counter
                        const uint32_t w = atomicAdd(wp.work_next, 1u);
                        if (w >= nchunks) {
                            done = true;
                        } else {
                            const uint32_t ck = wp.order ? wp.order[w] : w;
                            i = ck * wp.chunk;
                            range_end = (uint32_t)min((long long)n, (long long)i + wp.chunk);
                            if (i > 0 && i < range_end && diag_of(hits[i]) == diag_of(hits[i - 1]))
                                i = segment_end(hits, i, n, diag_of(hits[i]));
                            cur = i < n ? hits[i] : ~0ull;
                        }
                    } else {
                        done = true;
                    }
                }
                if (!done && i < range_end) {
                    D = diag_of(cur);
                    if (BATCH) seg_ctx<BATCH>(wp, D, c);
                    dq = (int)(c.qoff - (BATCH ? c.D : (long long)(D & 0x7FFFFFFFu)));
                    tr = (int)c.tlen - span;
                    qr = (int)c.qlen - span;
                    E = wp.Ecarry ? wp.Ecarry[D & 0x7FFFFFFFu] : INT_MIN;
                    in_seg = true;
                    handed = false;
                    cap = wp.lane_cap;
                    tasks++;
                }
            }
            if (in_seg) {
                t = (int)(uint32_t)cur;
                nxt = (i + 1 < n) ? hits[i + 1] : ~0ull;  // consumed when this hit is done
                if (t < E) {  // inside the last HSP of its diagonal: skipped
                    i++;
                    cur = nxt;
                } else {
                    q = t + dq;
                    ravail = min(tr - t, qr - q);
                    lavail = min(t, q);
                    R = LaneSide{0, 0, 0, 0, ravail == 0};
                    L = LaneSide{0, 0, 0, 0, lavail == 0};
                    busy = true;
                }
            }
        }
        if (__all_sync(0xffffffffu, done)) break;
        // (2) right sides
        const bool needR = busy && !R.done;
        if (__any_sync(0xffffffffu, needR) && needR)
            lane_window<PACKED, PLANES, !BATCH>(wp.T, c.Q, c.tb + t + span, c.qb + q + span, 1, ravail,
                                        X, lut, lut64, R, wp);
        // (3) left sides
        const bool needL = busy && !L.done;
        if (__any_sync(0xffffffffu, needL) && needL)
            lane_window<PACKED, PLANES, !BATCH>(wp.T, c.Q, c.tb + t, c.qb + q, -1, lavail, X, lut, lut64,
                                        L, wp);
        if (busy && (R.best > SCORE_LIMIT || L.best > SCORE_LIMIT)) status |= ST_SCORE_OVERFLOW;
        // (4) finish or hand off
        if (busy && R.done && L.done) {
            const long long rl = (long long)R.best + L.best;
            long long score = 0;
            bool pass = false;
            if (rl + s0_bound >= wp.thresh) {  // rare for random hits
                score = rl + span_score(wp.T, c.Q, c.tb + t, c.qb + q, span, psum, lut);
                if (score > INT_MAX) status |= ST_SCORE_OVERFLOW;
                pass = score >= wp.thresh;
            }
            ext++;
            cells += (unsigned long long)(span + R.n + L.n);
            log_ext(wp, c, t, q, R.n, L.n);
            if (pass) emit<BATCH>(wp, c, t, q, L.blen, R.blen, score, status);
            if (pass || !(wp.flags & SFE_SKIP_PASSING_ONLY)) E = (int)(t + span + R.blen);
            i++;
            cur = nxt;
            busy = false;
        } else if (busy && (R.n >= cap || L.n >= cap)) {
            // a long extension: the rest of this diagonal goes to a warp
            unsigned int slot = atomicAdd(wp.queue_len, 1u);
            if (slot < wp.queue_cap) {
                if (PERSIST) {
                    // entry first, then its epoch tag: a consumer that sees the tag sees the entry
                    wp.queue[slot].x = i;
                    wp.queue[slot].y = (uint32_t)E;
                    __threadfence();
                    atomicExch(&wp.queue[slot].z, wp.epoch);
                } else {
                    wp.queue[slot] = make_uint4(i, (uint32_t)E, 0u, 0u);
                }
                handed = true;
                shadow += (unsigned long long)(span + R.n + L.n);  // the warp scores it again
                i = segment_end(hits, i, n, D);
                cur = i < n ? hits[i] : ~0ull;
                in_seg = false;
                busy = false;
            } else {
                cap = INT_MAX;  // queue full: this lane finishes the diagonal itself
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ext += __shfl_down_sync(0xffffffffu, ext, o);
        cells += __shfl_down_sync(0xffffffffu, cells, o);
        tasks += __shfl_down_sync(0xffffffffu, tasks, o);
        shadow += __shfl_down_sync(0xffffffffu, shadow, o);
        status |= __shfl_down_sync(0xffffffffu, status, o);
    }
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        if (ext) atomicAdd(&wp.ctr->extended, ext);
        if (cells) atomicAdd(&wp.ctr->cells, cells);
        if (tasks) atomicAdd(&wp.ctr->lane_tasks, tasks);
        if (shadow) atomicAdd(&wp.ctr->shadow, shadow);
    }
    if (PERSIST) drain_queue<BATCH>(hits, n, wp, lut, lane, status);
    if (lane == 0 && status) atomicOr(&wp.ctr->status, status);
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

// The warp tier on one handed-off diagonal: from hit i with skip state E to
// the end of the diagonal, every extension in 32-base chunks.
template <bool BATCH>
__device__ void warp_walk_diagonal(const uint64_t *__restrict__ hits, uint32_t nhits, uint32_t i,
                                   int E, const WalkParams &wp, const int *lut, int lane,
                                   unsigned long long &ext, unsigned long long &cells,
                                   uint32_t &status) {
    const uint32_t dword = diag_of(hits[i]);
    SegCtx c;
    seg_ctx<BATCH>(wp, dword, c);
    const long long D = c.D;
    while (i < nhits) {
        const uint64_t h = hits[i];
        if (diag_of(h) != dword) break;
        const long long t = (long long)(uint32_t)h;
        if (t < E) {
            i++;
            continue;
        }
        const long long q = t - D + c.qoff;
        // seed span: lanes 0..span-1
        int s = 0;
        if (lane < wp.span)
            s = lut[base_at(wp.T, c.tb + t + lane) * 4u + base_at(c.Q, c.qb + q + lane)];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const long long pt = t + wp.span, pq = q + wp.span;
        const int ravail = (int)min(c.tlen - pt, c.qlen - pq);
        const int lavail = (int)min(t, q);
        const Side r = warp_side(wp.T, c.Q, c.tb + pt, c.qb + pq, +1, ravail, wp.xdrop, lut, lane,
                                 status);
        const Side l = warp_side(wp.T, c.Q, c.tb + t - 1, c.qb + q - 1, -1, lavail, wp.xdrop,
                                 lut, lane, status);
        const long long score = (long long)s + r.best + l.best;
        if (score > INT_MAX) status |= ST_SCORE_OVERFLOW;
        ext++;
        cells += (unsigned long long)(wp.span + r.scored + l.scored);
        if (lane == 0) log_ext(wp, c, t, q, r.scored, l.scored);
        const bool pass = score >= wp.thresh;
        if (pass && lane == 0) emit<BATCH>(wp, c, t, q, l.blen, r.blen, score, status);
        if (pass || !(wp.flags & SFE_SKIP_PASSING_ONLY)) E = (int)(t + wp.span + r.blen);
        i++;
    }
    if (wp.Ecarry && lane == 0) wp.Ecarry[D] = E;
}

// ---------------------------------------------------- speculative window
//
// The speculative batch of Algorithm 3, applied to the per-diagonal skip: a
// warp walks whole diagonals; on each, it takes the next K hits that the
// current skip state E does not already cover, extends them at once (group
// g of W = 32 / K lanes extends hit g in W-base chunks with group-wide
// shuffle scans), then commits the K results one by one in t order: a hit
// that an earlier committed extension now covers (t < E) is skipped and its
// work was shadow work (stats.shadow_cells); every other result is exactly
// the serial one, since an extension does not depend on E. K = 1 is the
// serial walk with one warp per hit.

template <int W>
__device__ __forceinline__ int grp_incl_sum(int v, int gl) {
#pragma unroll
    for (int o = 1; o < W; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o, W);
        if (gl >= o) v += y;
    }
    return v;
}

template <int W>
__device__ __forceinline__ int grp_incl_max(int v, int gl) {
#pragma unroll
    for (int o = 1; o < W; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o, W);
        if (gl >= o) v = max(v, y);
    }
    return v;
}

// One side of each group's hit (bases p0 + dir * k, k < avail) in chunks of W
// bases; every lane of a group returns its group's result. The loop runs
// until every group is done, so the shuffles always see the whole warp.
template <int W>
__device__ __forceinline__ Side group_side(const uint32_t *__restrict__ T,
                                           const uint32_t *__restrict__ Q, long long pt0,
                                           long long pq0, int dir, int avail, bool active, int X,
                                           const int *lut, int lane, uint32_t &status) {
    const int gl = lane & (W - 1), gbase = lane & ~(W - 1);
    const unsigned gmask = W == 32 ? 0xffffffffu : (((1u << W) - 1u) << gbase);
    int carry = 0, best = 0, blen = 0, scored = active ? avail : 0;
    bool done = !active || avail <= 0;
    for (int k0 = 0; __any_sync(0xffffffffu, !done); k0 += W) {
        const int k = k0 + gl;
        const bool valid = !done && k < avail;
        int s = 0;
        if (valid)
            s = lut[base_at(T, pt0 + dir * (long long)k) * 4u + base_at(Q, pq0 + dir * (long long)k)];
        const int P = grp_incl_sum<W>(s, gl) + carry;
        const int Mx = max(grp_incl_max<W>(P, gl), best);
        const unsigned stopm = __ballot_sync(0xffffffffu, valid && (Mx - P > X)) & gmask;
        const unsigned validm = __ballot_sync(0xffffffffu, valid) & gmask;
        const int nvalid = __popc(validm);
        const int last = stopm ? __ffs(stopm) - 1 - gbase : nvalid - 1;
        const int bl = __shfl_sync(0xffffffffu, Mx, gbase + max(0, last));
        const unsigned m =
            __ballot_sync(0xffffffffu, valid && gl <= last && P == bl) & gmask;
        const int cend = __shfl_sync(0xffffffffu, P, gbase + W - 1);
        if (!done) {
            if (bl > best) {
                blen = k0 + (__ffs(m) - 1 - gbase) + 1;
                best = bl;
            }
            if (best > SCORE_LIMIT) status |= ST_SCORE_OVERFLOW;
            if (stopm) {
                scored = k0 + last + 1;
                done = true;
            } else if (k0 + W >= avail) {
                done = true;
            }
            carry = cend;
        }
    }
    return {best, blen, scored};
}

template <int W, bool BATCH>
__global__ void __launch_bounds__(W_BLOCK) walk_spec_kernel(const uint64_t *__restrict__ hits,
                                                            uint32_t n, WalkParams wp) {
    constexpr int K = 32 / W;
    __shared__ int lut[16];
    if (threadIdx.x < 16) lut[threadIdx.x] = wp.scores[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane / W, gl = lane & (W - 1);
    const int span = wp.span, X = wp.xdrop;
    unsigned long long ext = 0, cells = 0, shadow = 0, tasks = 0;
    uint32_t status = 0;
    uint32_t nchunks = wp.nchunks;
    if (wp.nd) {  // the hit count lives on the device (n is the buffer's size)
        n = (uint32_t)min((unsigned long long)n, *wp.nd);
        nchunks = (n + wp.chunk - 1) / wp.chunk;
    }
    SegCtx c;
    seg_ctx<BATCH>(wp, 0u, c);
    while (true) {
        uint32_t w = 0;
        if (lane == 0) w = atomicAdd(wp.work_next, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= nchunks) break;
        uint32_t i = w * wp.chunk;
        const uint32_t end = (uint32_t)min((long long)n, (long long)i + wp.chunk);
        // a diagonal that started before this chunk belongs to the previous one
        if (i > 0 && i < end && diag_of(hits[i]) == diag_of(hits[i - 1]))
            i = segment_end(hits, i, n, diag_of(hits[i]));
        while (i < end) {
            const uint32_t D = diag_of(hits[i]);
            const uint32_t se = segment_end(hits, i, n, D);
            if (BATCH) seg_ctx<BATCH>(wp, D, c);  // the diagonal's pair and strand
            const long long Dl = BATCH ? c.D : (long long)(D & 0x7FFFFFFFu);
            const long long qoff = c.qoff;
            int E = wp.Ecarry ? wp.Ecarry[Dl] : INT_MIN;
            tasks++;
            uint32_t j = i;
            while (true) {
                while (j < se && (long long)(uint32_t)hits[j] < E) j++;  // covered: skipped
                if (j >= se) break;
                // the window: hits j .. j + K - 1 of this diagonal, group g takes j + g
                const uint32_t my = j + g;
                const bool active = my < se;
                const long long t = active ? (long long)(uint32_t)hits[my] : 0;
                const long long q = t - Dl + qoff;
                int s = 0;
                if (active)
                    for (int k = gl; k < span; k += W)
                        s += lut[base_at(wp.T, c.tb + t + k) * 4u + base_at(c.Q, c.qb + q + k)];
                s = grp_incl_sum<W>(s, gl);
                const int s0 = __shfl_sync(0xffffffffu, s, (lane & ~(W - 1)) + W - 1);
                const int ravail = active ? (int)min(c.tlen - t - span, c.qlen - q - span) : 0;
                const int lavail = active ? (int)min(t, q) : 0;
                const Side r = group_side<W>(wp.T, c.Q, c.tb + t + span, c.qb + q + span, +1,
                                             ravail, active, X, lut, lane, status);
                const Side l = group_side<W>(wp.T, c.Q, c.tb + t - 1, c.qb + q - 1, -1, lavail,
                                             active, X, lut, lane, status);
                // commit in t order
                for (int gg = 0; gg < K && j + gg < se; gg++) {
                    const int src = gg * W;
                    const long long tg = __shfl_sync(0xffffffffu, t, src);
                    const long long qg = __shfl_sync(0xffffffffu, q, src);
                    const int sg = __shfl_sync(0xffffffffu, s0, src);
                    const int rb = __shfl_sync(0xffffffffu, r.best, src);
                    const int rbl = __shfl_sync(0xffffffffu, r.blen, src);
                    const int rsc = __shfl_sync(0xffffffffu, r.scored, src);
                    const int lb = __shfl_sync(0xffffffffu, l.best, src);
                    const int lbl = __shfl_sync(0xffffffffu, l.blen, src);
                    const int lsc = __shfl_sync(0xffffffffu, l.scored, src);
                    const unsigned long long work = (unsigned long long)(span + rsc + lsc);
                    if (tg < E) {  // covered by a hit committed in this window
                        shadow += work;
                        continue;
                    }
                    const long long score = (long long)sg + rb + lb;
                    if (score > INT_MAX) status |= ST_SCORE_OVERFLOW;
                    ext++;
                    cells += work;
                    if (lane == 0) log_ext(wp, c, tg, qg, rsc, lsc);
                    const bool pass = score >= wp.thresh;
                    if (pass && lane == 0) emit<BATCH>(wp, c, tg, qg, lbl, rbl, score, status);
                    if (pass || !(wp.flags & SFE_SKIP_PASSING_ONLY)) E = (int)(tg + span + rbl);
                }
                j += K;
            }
            if (wp.Ecarry && lane == 0) wp.Ecarry[Dl] = E;
            i = se;
        }
    }
    if (lane == 0) {
        if (ext) atomicAdd(&wp.ctr->extended, ext);
        if (cells) atomicAdd(&wp.ctr->cells, cells);
        if (shadow) atomicAdd(&wp.ctr->shadow, shadow);
        if (tasks) atomicAdd(&wp.ctr->warp_tasks, tasks);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) status |= __shfl_down_sync(0xffffffffu, status, o);
    if (lane == 0 && status) atomicOr(&wp.ctr->status, status);
}

template <bool BATCH>
__global__ void __launch_bounds__(W_BLOCK) walk_warps_kernel(const uint64_t *__restrict__ hits,
                                                             uint32_t nhits, WalkParams wp) {
    __shared__ int lut[16];
    if (threadIdx.x < 16) lut[threadIdx.x] = wp.scores[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const unsigned long long nq = min((unsigned long long)*wp.queue_len, wp.queue_cap);
    if (wp.nd) nhits = (uint32_t)min((unsigned long long)nhits, *wp.nd);
    unsigned long long ext = 0, cells = 0, tasks = 0;
    uint32_t status = 0;
    for (long long e = warp; e < (long long)nq; e += nwarps) {
        const uint4 it = wp.queue[e];
        // after a persistent walk: only the entries its consumers left (a slot
        // reserved but never published is skipped: it holds no task)
        if (wp.deferred_only && (it.z != wp.epoch || it.w == wp.epoch)) continue;
        tasks++;
        warp_walk_diagonal<BATCH>(hits, nhits, it.x, (int)it.y, wp, lut, lane, ext, cells, status);
    }
    if (lane == 0) {
        if (ext) atomicAdd(&wp.ctr->extended, ext);
        if (cells) {
            atomicAdd(&wp.ctr->cells, cells);
            atomicAdd(&wp.ctr->warp_cells, cells);
        }
        if (tasks) atomicAdd(&wp.ctr->warp_tasks, tasks);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) status |= __shfl_down_sync(0xffffffffu, status, o);
    if (lane == 0 && status) atomicOr(&wp.ctr->status, status);
}

inline unsigned grid_for(long long n, int block = BLOCK) {
    return (unsigned)((n + block - 1) / block);
}

int sms() { return device_sms(); }

}  // namespace

cudaError_t launch_walk_lanes(const uint64_t *hits, long long n, WalkParams wp, int lanes_per_sm,
                              cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    // about two resident waves of lanes, each owning a contiguous hit range
    long long lanes = (long long)sms() * (lanes_per_sm > 0 ? lanes_per_sm : 4096);
    long long chunk = (n + lanes - 1) / lanes;
    if (chunk < 16) chunk = 16;
    long long nthreads = (n + chunk - 1) / chunk;
    g_launches++;
    const unsigned grid = grid_for(nthreads, W_BLOCK);
    const bool packed = wp.xdrop < PACKED_X_LIMIT, batch = wp.pairs != nullptr;
    if (packed && !batch && wp.TN)
        walk_lanes_kernel<true, false, false, true><<<grid, W_BLOCK, 0, st>>>(hits, (uint32_t)n, (uint32_t)chunk, wp);
    else if (packed && !batch)
        walk_lanes_kernel<true, false, false><<<grid, W_BLOCK, 0, st>>>(hits, (uint32_t)n, (uint32_t)chunk, wp);
    else if (!packed && !batch)
        walk_lanes_kernel<false, false, false><<<grid, W_BLOCK, 0, st>>>(hits, (uint32_t)n, (uint32_t)chunk, wp);
    else if (packed)
        walk_lanes_kernel<true, true, false><<<grid, W_BLOCK, 0, st>>>(hits, (uint32_t)n, (uint32_t)chunk, wp);
    else
        walk_lanes_kernel<false, true, false><<<grid, W_BLOCK, 0, st>>>(hits, (uint32_t)n, (uint32_t)chunk, wp);
    return cudaGetLastError();
}

cudaError_t launch_walk_warps(const uint64_t *hits, long long n, WalkParams wp, int grid_warps,
                              cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (grid_warps <= 0) grid_warps = 8 * sms() * (W_BLOCK / 32);
    unsigned grid = (unsigned)((grid_warps * 32 + W_BLOCK - 1) / W_BLOCK);
    g_launches++;
    if (wp.pairs)
        walk_warps_kernel<true><<<grid, W_BLOCK, 0, st>>>(hits, (uint32_t)n, wp);
    else
        walk_warps_kernel<false><<<grid, W_BLOCK, 0, st>>>(hits, (uint32_t)n, wp);
    return cudaGetLastError();
}

// Sort key of each work chunk for the largest-first schedule: the number of
// hits of the diagonal its first hit lies on (descending), then chunk index.
// Keys of the chunk schedules (sorted ascending by their high word). Chunks
// past a device-side hit count (nd) get the largest key, so the ones that
// exist come first.
__global__ void chunk_keys_kernel(const uint64_t *__restrict__ hits, uint32_t n,
                                  const unsigned long long *nd, uint32_t chunk, uint32_t nchunks,
                                  int random, uint64_t *__restrict__ keys) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nchunks) return;
    if (nd) n = (uint32_t)min((unsigned long long)n, *nd);
    if ((unsigned long long)k * chunk >= n) {
        keys[k] = (0xFFFFFFFFull << 32) | k;
        return;
    }
    if (random) {  // a fixed pseudo-random order (splitmix64 finaliser of k)
        unsigned long long z = 0x9E3779B97F4A7C15ull * (unsigned long long)(k + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        keys[k] = (z & 0x7FFFFFFF00000000ull) | k;
        return;
    }
    const uint32_t i = k * chunk;
    const uint32_t d = diag_of(hits[i]);
    uint32_t lo = 0, hi = i;  // first index of this diagonal
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (diag_of(hits[mid]) < d)
            lo = mid + 1;
        else
            hi = mid;
    }
    const uint32_t len = segment_end(hits, i, n, d) - lo;
    keys[k] = ((uint64_t)(0xFFFFFFFFu - len) << 32) | k;
}

__global__ void chunk_order_kernel(const uint64_t *__restrict__ keys, uint32_t nchunks,
                                   uint32_t *__restrict__ order) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nchunks) order[k] = (uint32_t)keys[k];
}

template <bool PACKED, bool BATCH, bool PLANES = false>
cudaError_t launch_persistent_t(const uint64_t *hits, long long n, const WalkParams &wp,
                                cudaStream_t st) {
    // every CTA resident at once: consumers wait on producers of other CTAs
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, walk_lanes_kernel<PACKED, BATCH, true, PLANES>, W_BLOCK, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    g_launches++;
    walk_lanes_kernel<PACKED, BATCH, true, PLANES><<<per_sm * sms(), W_BLOCK, 0, st>>>(
        hits, (uint32_t)n, wp.chunk, wp);
    return cudaGetLastError();
}

uint32_t walk_auto_chunk(long long n) {
    // about 16 chunks per resident lane (4 CTAs of W_BLOCK per SM), 16 to 256
    // hits (measured: 100 Mb pair tiles of ~1e9 hits walk 1.6% faster with
    // 256 than with 64, the 10 Mb pair slower with 81 than with 32-64, and a
    // 3 Mb pair needs 16 for the counter to balance the lanes)
    const long long lanes = 4LL * sms() * W_BLOCK;
    const long long c = (n + 16 * lanes - 1) / (16 * lanes);
    return (uint32_t)(c < 16 ? 16 : (c > 256 ? 256 : c));
}

cudaError_t launch_walk_persistent(const uint64_t *hits, long long n, WalkParams wp,
                                   cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (wp.chunk == 0) wp.chunk = walk_auto_chunk(n);
    wp.nchunks = (uint32_t)((n + wp.chunk - 1) / wp.chunk);
    const bool packed = wp.xdrop < PACKED_X_LIMIT, batch = wp.pairs != nullptr;
    if (packed && !batch && wp.TN) return launch_persistent_t<true, false, true>(hits, n, wp, st);
    if (packed && !batch) return launch_persistent_t<true, false>(hits, n, wp, st);
    if (!packed && !batch) return launch_persistent_t<false, false>(hits, n, wp, st);
    if (packed) return launch_persistent_t<true, true>(hits, n, wp, st);
    return launch_persistent_t<false, true>(hits, n, wp, st);
}

template <bool BATCH>
static cudaError_t launch_spec(const uint64_t *hits, uint32_t n, const WalkParams &wp, int window,
                               unsigned grid, cudaStream_t st) {
    switch (window) {
    case 1: walk_spec_kernel<32, BATCH><<<grid, W_BLOCK, 0, st>>>(hits, n, wp); break;
    case 2: walk_spec_kernel<16, BATCH><<<grid, W_BLOCK, 0, st>>>(hits, n, wp); break;
    case 4: walk_spec_kernel<8, BATCH><<<grid, W_BLOCK, 0, st>>>(hits, n, wp); break;
    case 8: walk_spec_kernel<4, BATCH><<<grid, W_BLOCK, 0, st>>>(hits, n, wp); break;
    case 16: walk_spec_kernel<2, BATCH><<<grid, W_BLOCK, 0, st>>>(hits, n, wp); break;
    default: walk_spec_kernel<1, BATCH><<<grid, W_BLOCK, 0, st>>>(hits, n, wp); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_walk_speculative(const uint64_t *hits, long long n, WalkParams wp, int window,
                                    cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (wp.chunk == 0) wp.chunk = walk_auto_chunk(n);
    wp.nchunks = (uint32_t)((n + wp.chunk - 1) / wp.chunk);
    const unsigned grid = (unsigned)(4 * sms());
    if (window != 1 && window != 2 && window != 4 && window != 8 && window != 16 && window != 32)
        return cudaErrorInvalidValue;
    g_launches++;
    if (wp.pairs)
        return launch_spec<true>(hits, (uint32_t)n, wp, window, grid, st);
    return launch_spec<false>(hits, (uint32_t)n, wp, window, grid, st);
}

size_t walk_schedule_temp_bytes(long long n, uint32_t chunk) {
    const long long nchunks = (n + chunk - 1) / chunk;
    return (size_t)nchunks * 20 + radix_sort_temp_bytes(nchunks) + 1024;
}

cudaError_t launch_walk_schedule(const uint64_t *hits, long long n, const WalkParams &wp,
                                 int schedule, const void *model, void *tmp, uint32_t **order,
                                 uint32_t *status, cudaStream_t st) {
    *order = nullptr;
    const uint32_t chunk = wp.chunk;
    if (schedule == SFE_SCHED_NATURAL || n <= 0) return cudaSuccess;
    const uint32_t nchunks = (uint32_t)((n + chunk - 1) / chunk);
    char *p = reinterpret_cast<char *>(tmp);
    uint64_t *ka = reinterpret_cast<uint64_t *>(p);
    uint64_t *kb = ka + ((nchunks + 31) & ~31u);
    uint32_t *ord = reinterpret_cast<uint32_t *>(kb + ((nchunks + 31) & ~31u));
    void *rt = ord + ((nchunks + 63) & ~63u);
    if (schedule == SFE_SCHED_PREDICTED) {
        cudaError_t e0 = launch_chunk_predict(hits, n, chunk, nchunks, wp, model, ka, st);
        if (e0 != cudaSuccess) return e0;
    } else {
        g_launches++;
        chunk_keys_kernel<<<grid_for(nchunks), BLOCK, 0, st>>>(
            hits, (uint32_t)n, wp.nd, chunk, nchunks, schedule == SFE_SCHED_RANDOM ? 1 : 0, ka);
    }
    bool in_b = false;
    cudaError_t e = radix_sort(ka, kb, nullptr, nullptr, nchunks, 32, 64, rt, &in_b, status, st);
    if (e != cudaSuccess) return e;
    g_launches++;
    chunk_order_kernel<<<grid_for(nchunks), BLOCK, 0, st>>>(in_b ? kb : ka, nchunks, ord);
    *order = ord;
    return cudaGetLastError();
}

}  // namespace sfe
