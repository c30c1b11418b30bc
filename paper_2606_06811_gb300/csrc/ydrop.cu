// Gapped Y-drop extension (the extension stage after the filter: Algorithm 1's
// YDropExtension, run in Algorithm 3's speculative batches).
//
// One warp per anchor half (forward or backward from the anchor), as the
// paper's systolic kernel maps one anchor-half per block. The affine-gap
// dynamic program is evaluated by anti-diagonals d = i + j: cell (i, j) has
// consumed i target and j query bases. The warp keeps the last two
// anti-diagonals in shared memory slots of at most `band` cells (H of d - 2,
// d - 1 and d; E and F only of d - 1 and d: 7 KB per warp at band 256, so 8
// CTAs of 4 warps fit an SM where 9 slots allowed 6: 182 -> 189 GCUPS); lanes
// take the cells of anti-diagonal d in chunks of 32, each reading its
// diagonal predecessor from d - 2 and its two gap predecessors from d - 1.
// Each lane keeps its live rows and its first best cell over the chunks, and
// four warp reductions per anti-diagonal give the live range and the best
// cell. A cell is live while H >= best - Y (best over the earlier
// anti-diagonals); anti-diagonal d computes every cell from the lowest to the
// highest i next to a live cell of d - 1 or one diagonal step from a live cell
// of d - 2, at most `band` of them, and the half stops after two
// anti-diagonals without a live cell. Same rule, same cells, same result as
// the oracle's or_ydrop_half.
//
// Small batches use ydrop_coop_kernel below (a CTA of cooperative warps per
// anchor half) with the same helpers and the same result.
//
// (Measured and not kept: the two anti-diagonals in registers, lane L holding
// rows base + 32 r + L of a sliding window and passing row i - 1 to lane L + 1
// by a rotation shuffle, as in the paper's shuffle-systolic kernel: 124
// registers and 4 CTAs per SM, 142 against 156 GCUPS.)
#include <climits>

#include "sfe_internal.cuh"

namespace sfe {

namespace {

constexpr int YD_WARPS = 4;        // warps per CTA (each owns 7 * band ints of shared memory)
constexpr int YD_NEG = -(1 << 29); // -inf that survives subtracting a gap cost
constexpr int YD_LIMIT = 1 << 30;  // a score above this flags overflow

struct YdSlot {
    int *H, *E, *F;
};

// The sequences of one anchor half. The base consumed by step i (1-based) is
// word (o >> 4), bits 2 (o & 15) of Tw (Qw) with o = tc + ts * i (qc + ts * j):
// forward, position p0 + i - 1; backward, p0 - i (o may then be negative, and
// >> and & floor it). TL, QL: bases the half may consume on each sequence.
struct YdSeq {
    const uint32_t *Tw, *Qw;
    int tc, qc, ts;
    long long TL, QL;
};

__device__ __forceinline__ YdSeq yd_seq(const uint32_t *T, long long tlen, const uint32_t *Qp,
                                        const uint32_t *Qm, long long qlen, int4 a, int dir) {
    YdSeq sq;
    const uint32_t *Q = a.x ? Qm : Qp;
    const long long t0 = a.y, q0 = a.z;
    sq.TL = dir > 0 ? tlen - t0 : t0;
    sq.QL = dir > 0 ? qlen - q0 : q0;
    sq.ts = dir;
    sq.Tw = T + (t0 >> 4);
    sq.Qw = Q + (q0 >> 4);
    sq.tc = (int)(t0 & 15) - (dir > 0 ? 1 : 0);
    sq.qc = (int)(q0 & 15) - (dir > 0 ? 1 : 0);
    return sq;
}

// Rows of anti-diagonal d to compute, from the live rows of d - 1 (L1..R1)
// and d - 2 (L2..R2; L > R: none), clipped to the sequences and the band.
__device__ __forceinline__ void yd_range(long long L1, long long R1, long long L2, long long R2,
                                         long long d, const YdSeq &sq, int band, long long &clo,
                                         long long &chi) {
    if (L1 <= R1 && L2 <= R2) {
        clo = min(L1, L2 + 1);
        chi = max(R1 + 1, R2 + 1);
    } else if (L1 <= R1) {
        clo = L1;
        chi = R1 + 1;
    } else {
        clo = L2 + 1;
        chi = R2 + 1;
    }
    clo = max(clo, max(0LL, d - sq.QL));
    chi = min(min(chi, sq.TL), d);
    chi = min(chi, clo + band - 1);
}

// The slots of one anti-diagonal addressed by row: H2m[i] is H of row i - 1
// on d - 2, H1o / E1o [i] row i on d - 1, H1m / F1m [i] row i - 1 on d - 1,
// H0 / E0 / F0 [i] row i on d; with the computed ranges of d - 1 and d - 2
// (first row and width) for the range checks. 32-bit rows and pointers set
// once per anti-diagonal: 13% fewer instructions than 64-bit rows and offsets
// per cell (156 -> 179 GCUPS). An empty range gets a first row no i reaches.
struct YdRows {
    const int *H2m, *H1o, *E1o, *H1m, *F1m;
    int *H0, *E0, *F0;
    int l1, w1, l2, w2;
};

__device__ __forceinline__ YdRows yd_rows(const YdSlot &c0, const YdSlot &c1, const YdSlot &c2,
                                          long long lo1, long long hi1, long long lo2,
                                          long long hi2, int ilo) {
    YdRows r;
    const bool e1 = lo1 > hi1, e2 = lo2 > hi2;
    r.l1 = e1 ? -(1 << 30) : (int)lo1;
    r.w1 = e1 ? 0 : (int)(hi1 - lo1);
    r.l2 = e2 ? -(1 << 30) : (int)lo2;
    r.w2 = e2 ? 0 : (int)(hi2 - lo2);
    r.H2m = e2 ? c2.H : c2.H - r.l2 - 1;
    r.H1o = e1 ? c1.H : c1.H - r.l1;
    r.E1o = e1 ? c1.E : c1.E - r.l1;
    r.H1m = e1 ? c1.H : c1.H - r.l1 - 1;
    r.F1m = e1 ? c1.F : c1.F - r.l1 - 1;
    r.H0 = c0.H - ilo;
    r.E0 = c0.E - ilo;
    r.F0 = c0.F - ilo;
    return r;
}

// Cell (i, j) of the current anti-diagonal: the affine recurrences, the
// Y-drop test (dead below floor_h), and H, E, F stored in the slots of d.
// Returns H (YD_NEG: dead).
__device__ __forceinline__ int yd_cell(const YdRows &r, const YdSeq &sq, int i, int j,
                                       const int *lut, int go, int ge, int floor_h) {
    int dg = YD_NEG, e = YD_NEG, f = YD_NEG;
    if (j >= 1 && (unsigned)(i - 1 - r.l2) <= (unsigned)r.w2) {
        const int hp = r.H2m[i];
        if (hp > YD_NEG) {
            const int ot = sq.tc + sq.ts * i, oq = sq.qc + sq.ts * j;
            const int bt = (int)((__ldg(sq.Tw + (ot >> 4)) >> ((ot & 15) * 2)) & 3u);
            const int bq = (int)((__ldg(sq.Qw + (oq >> 4)) >> ((oq & 15) * 2)) & 3u);
            dg = hp + lut[bt * 4 + bq];
        }
    }
    if (j >= 1 && (unsigned)(i - r.l1) <= (unsigned)r.w1) {
        const int hp = r.H1o[i];
        if (hp > YD_NEG) e = max(r.E1o[i] - ge, hp - go - ge);
    }
    if ((unsigned)(i - 1 - r.l1) <= (unsigned)r.w1) {
        const int hp = r.H1m[i];
        if (hp > YD_NEG) f = max(r.F1m[i] - ge, hp - go - ge);
    }
    int h = max(dg, max(e, f));
    if (h < floor_h) h = e = f = YD_NEG;
    r.H0[i] = h;
    r.E0[i] = e;
    r.F0[i] = f;
    return h;
}

__global__ void __launch_bounds__(YD_WARPS * 32) ydrop_half_kernel(
    const uint32_t *__restrict__ T, long long tlen, const uint32_t *__restrict__ Qp,
    const uint32_t *__restrict__ Qm, long long qlen, const int4 *__restrict__ anchors,
    int ntasks, YdParams prm, YdHalf *__restrict__ out) {
    extern __shared__ int yd_smem[];
    __shared__ int lut[16];
    if (threadIdx.x < 16) lut[threadIdx.x] = prm.scores[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int task = blockIdx.x * YD_WARPS + wib;
    if (task >= ntasks) return;  // whole warp
    const int band = prm.band;
    // H of three anti-diagonals (d, d - 1, d - 2), E and F of two (d, d - 1)
    int *wbuf = yd_smem + wib * 7 * band;
    auto slot = [&](int s, int k) {
        return YdSlot{wbuf + s * band, wbuf + (3 + k) * band, wbuf + (5 + k) * band};
    };
    const YdSeq sq = yd_seq(T, tlen, Qp, Qm, qlen, anchors[task >> 1], (task & 1) ? -1 : 1);
    const int go = prm.gap_open, ge = prm.gap_extend, Y = prm.ydrop;
    // anti-diagonal 0: the origin in slot 1 (d - 1); slot 2 (d - 2) empty
    int s0 = 0, s1 = 1, s2 = 2, k0 = 0, k1 = 1;
    if (lane == 0) {
        slot(s1, k1).H[0] = 0;
        slot(s1, k1).E[0] = YD_NEG;
        slot(s1, k1).F[0] = YD_NEG;
    }
    __syncwarp();
    long long lo1 = 0, hi1 = 0, L1 = 0, R1 = 0, lo2 = 1, hi2 = 0, L2 = 1, R2 = 0;
    long long best = 0, cells = 0;
    int bi = 0, bj = 0;
    uint32_t status = 0;
    for (long long d = 1;; d++) {
        if (L1 > R1 && L2 > R2) break;
        long long clo, chi;
        yd_range(L1, R1, L2, R2, d, sq, band, clo, chi);
        // the lane's live rows and first best cell, combined over the warp once
        // per anti-diagonal: a ballot and a reduction per chunk put a
        // warp-wide dependency between the chunks (measured on the 10 Mb
        // pair's anchors, batch 16,384: 126 against 156 GCUPS)
        int lfirst = INT_MAX, llast = -1, lbest = YD_NEG, lrow = INT_MAX;
        // a cell is dead below this (best - Y, or at most YD_NEG: no predecessor)
        const int floor_h = (int)max(best - Y, (long long)YD_NEG + 1);
        const int ilo = (int)clo, ihi = (int)chi;
        const YdRows rows = yd_rows(slot(s0, k0), slot(s1, k1), slot(s2, k0), lo1, hi1, lo2, hi2,
                                    ilo);  // the third slot: its H only
        const int d32 = (int)d;  // j = d - i in 32 bits (exact: j < 2^31)
        for (int b = ilo; b <= ihi; b += 32) {
            const int i = b + lane, j = d32 - i;
            const int h = i <= ihi ? yd_cell(rows, sq, i, j, lut, go, ge, floor_h) : YD_NEG;
            if (h > YD_NEG) {  // chunks in increasing rows: the lane's first best
                if (lfirst == INT_MAX) lfirst = i;
                llast = i;
                if (h > lbest) {
                    lbest = h;
                    lrow = i;
                }
            }
        }
        const int dbest = __reduce_max_sync(0xffffffffu, lbest);
        long long L0 = 1, R0 = 0, dbi = 0;
        if (dbest > YD_NEG) {
            dbi = __reduce_min_sync(0xffffffffu, lbest == dbest ? lrow : INT_MAX);
            L0 = __reduce_min_sync(0xffffffffu, lfirst);
            R0 = __reduce_max_sync(0xffffffffu, llast);
        }
        if (clo <= chi) cells += chi - clo + 1;
        __syncwarp();  // this anti-diagonal's cells are written before the next reads them
        if (dbest > best) {
            best = dbest;
            bi = (int)dbi;
            bj = (int)(d - dbi);
            if (best > YD_LIMIT) status |= ST_SCORE_OVERFLOW;
        }
        const int sfree = s2;
        s2 = s1;
        s1 = s0;
        s0 = sfree;
        const int kf = k1;
        k1 = k0;
        k0 = kf;
        lo2 = lo1;
        hi2 = hi1;
        L2 = L1;
        R2 = R1;
        lo1 = clo;
        hi1 = chi;
        L1 = L0;
        R1 = R0;
        if (clo > chi) {
            lo1 = 1;
            hi1 = 0;
        }
    }
    if (lane == 0) {
        YdHalf r;
        r.best = (int)best;
        r.bi = bi;
        r.bj = bj;
        r.status = status;
        r.cells = cells;
        out[task] = r;
    }
}

// The same extension with a CTA of YC_WARPS warps per anchor half, for
// batches too small to fill the GPU with one warp per half (the paper's
// Section 8: cooperative warps per anchor half raise the occupancy of small
// speculative batches). Warp w computes rows clo + 32 w .. clo + 32 w + 31 of
// each anti-diagonal (the band is at most YC_WARPS chunks); each warp reduces
// its live rows and first best cell, one barrier per anti-diagonal publishes
// the slots and the partial results, and every thread combines the partials
// in warp order (lower rows first), so all warps hold the same state. Same
// cells, same result as the warp kernel.
constexpr int YC_WARPS = YD_MAX_BAND / 32;
constexpr int YC_MAX_TASKS_PER_SM = 16;  // two waves of the 8 CTAs an SM holds (batch 1024: 1721 -> 1629 ms)

__global__ void __launch_bounds__(YC_WARPS * 32, 8) ydrop_coop_kernel(
    const uint32_t *__restrict__ T, long long tlen, const uint32_t *__restrict__ Qp,
    const uint32_t *__restrict__ Qm, long long qlen, const int4 *__restrict__ anchors,
    YdParams prm, YdHalf *__restrict__ out) {
    __shared__ int lut[16];
    __shared__ int slots[7 * YD_MAX_BAND];
    __shared__ int part[2][YC_WARPS][4];  // per warp: best, its first row, first / last live row
    if (threadIdx.x < 16) lut[threadIdx.x] = prm.scores[threadIdx.x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int task = blockIdx.x;  // one anchor half per CTA: the grid is the task count
    const int band = prm.band;
    auto slot = [&](int s, int k) {
        return YdSlot{slots + s * band, slots + (3 + k) * band, slots + (5 + k) * band};
    };
    const YdSeq sq = yd_seq(T, tlen, Qp, Qm, qlen, anchors[task >> 1], (task & 1) ? -1 : 1);
    const int go = prm.gap_open, ge = prm.gap_extend, Y = prm.ydrop;
    int s0 = 0, s1 = 1, s2 = 2, k0 = 0, k1 = 1;
    if (threadIdx.x == 0) {
        slot(s1, k1).H[0] = 0;
        slot(s1, k1).E[0] = YD_NEG;
        slot(s1, k1).F[0] = YD_NEG;
    }
    __syncthreads();
    long long lo1 = 0, hi1 = 0, L1 = 0, R1 = 0, lo2 = 1, hi2 = 0, L2 = 1, R2 = 0;
    long long best = 0, cells = 0;
    int bi = 0, bj = 0, par = 0;
    uint32_t status = 0;
    for (long long d = 1;; d++) {
        if (L1 > R1 && L2 > R2) break;  // the same decision in every thread
        long long clo, chi;
        yd_range(L1, R1, L2, R2, d, sq, band, clo, chi);
        const int floor_h = (int)max(best - Y, (long long)YD_NEG + 1);
        const int ilo = (int)clo, ihi = (int)chi;
        const YdRows rows = yd_rows(slot(s0, k0), slot(s1, k1), slot(s2, k0), lo1, hi1, lo2, hi2,
                                    ilo);
        int lfirst = INT_MAX, llast = -1, lbest = YD_NEG, lrow = INT_MAX;
        {
            const int i = ilo + 32 * w + lane, j = (int)d - i;
            const int h = i <= ihi ? yd_cell(rows, sq, i, j, lut, go, ge, floor_h) : YD_NEG;
            if (h > YD_NEG) {
                lfirst = llast = lrow = i;
                lbest = h;
            }
        }
        const int wb = __reduce_max_sync(0xffffffffu, lbest);
        const int wr = __reduce_min_sync(0xffffffffu, lbest == wb ? lrow : INT_MAX);
        const int wf = __reduce_min_sync(0xffffffffu, lfirst);
        const int wl = __reduce_max_sync(0xffffffffu, llast);
        if (lane == 0) {
            part[par][w][0] = wb;
            part[par][w][1] = wr;
            part[par][w][2] = wf;
            part[par][w][3] = wl;
        }
        __syncthreads();  // the anti-diagonal's cells and partials are published
        int dbest = YD_NEG, dbi = 0, L0 = INT_MAX, R0 = -1;
#pragma unroll
        for (int k = 0; k < YC_WARPS; k++) {  // warps in increasing rows: the first best
            const int b = part[par][k][0];
            if (b > dbest) {
                dbest = b;
                dbi = part[par][k][1];
            }
            L0 = min(L0, part[par][k][2]);
            R0 = max(R0, part[par][k][3]);
        }
        par ^= 1;  // the next anti-diagonal writes the other partials
        if (clo <= chi) cells += chi - clo + 1;
        if (dbest > best) {
            best = dbest;
            bi = dbi;
            bj = (int)(d - dbi);
            if (best > YD_LIMIT) status |= ST_SCORE_OVERFLOW;
        }
        const int sfree = s2;
        s2 = s1;
        s1 = s0;
        s0 = sfree;
        const int kf = k1;
        k1 = k0;
        k0 = kf;
        lo2 = lo1;
        hi2 = hi1;
        L2 = L1;
        R2 = R1;
        lo1 = clo;
        hi1 = chi;
        if (dbest > YD_NEG) {
            L1 = L0;
            R1 = R0;
        } else {
            L1 = 1;
            R1 = 0;
        }
        if (clo > chi) {
            lo1 = 1;
            hi1 = 0;
        }
    }
    if (threadIdx.x == 0) {
        YdHalf r;
        r.best = (int)best;
        r.bi = bi;
        r.bj = bj;
        r.status = status;
        r.cells = cells;
        out[task] = r;
    }
}

}  // namespace

size_t ydrop_smem_bytes(int band) { return (size_t)YD_WARPS * 7 * band * sizeof(int); }

cudaError_t launch_ydrop(const uint32_t *T, long long tlen, const uint32_t *Qp,
                         const uint32_t *Qm, long long qlen, const int4 *anchors, int nanchors,
                         const YdParams &prm, YdHalf *out, cudaStream_t st) {
    if (nanchors <= 0) return cudaSuccess;
    const size_t smem = ydrop_smem_bytes(prm.band);
    static std::atomic<unsigned long long> attr;
    cudaError_t e = once_per_device(attr, [] {
        return cudaFuncSetAttribute(ydrop_half_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)ydrop_smem_bytes(YD_MAX_BAND));
    });
    if (e != cudaSuccess) return e;
    const int ntasks = 2 * nanchors;
    g_launches++;
    if (ntasks <= YC_MAX_TASKS_PER_SM * device_sms()) {
        // too few halves to fill the GPU a warp each: a CTA per half
        ydrop_coop_kernel<<<(unsigned)ntasks, YC_WARPS * 32, 0, st>>>(T, tlen, Qp, Qm, qlen,
                                                                       anchors, prm, out);
        return cudaGetLastError();
    }
    const unsigned grid = (unsigned)((ntasks + YD_WARPS - 1) / YD_WARPS);
    ydrop_half_kernel<<<grid, YD_WARPS * 32, smem, st>>>(T, tlen, Qp, Qm, qlen, anchors, ntasks,
                                                         prm, out);
    return cudaGetLastError();
}

}  // namespace sfe
