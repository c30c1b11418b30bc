// C ABI of libsfe (declared in include/sfe.h): context and scratch arena,
// host/device staging, and the order of the kernels of the filter stage.
#include <algorithm>
#include <chrono>
#include <unordered_map>
#include <climits>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sfe_internal.cuh"

using namespace sfe;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define CK(x)                                                                              \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            return fail(SFE_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_));       \
        }                                                                                  \
    } while (0)

#define TRY(x)                   \
    do {                         \
        int r_ = (x);            \
        if (r_ != SFE_OK) return r_; \
    } while (0)

// HOXD70 (Chiaromonte, Yap and Miller 2002), target base major, order ACGT.
const int32_t kHoxd70[16] = {91,   -114, -31, -123, -114, 100,  -125, -31,
                             -31,  -125, 100, -114, -123, -31,  -114, 91};
const char *kDefaultPattern = "1110100110010101111";

constexpr long long kDefaultTileHits = 1LL << 30;  // 8 GB per hit buffer
constexpr unsigned long long kQueueMax = 1ull << 20;
// A batch pair's split-key tables have about npos / 2 buckets each (1 to 2
// entries per bucket: measured on 4096 pairs, 20.6 ms per batch against 21.2
// with one bucket per position and 21.2 / 23.8 with 4 / 8 per bucket).
constexpr int kBatchBucketShift = 1;
// Cell planes of a single pair (half a byte per base of T and of each query
// strand) are built up to half of the GB300's 126 MB L2.
constexpr size_t kPlanesMaxBytes = 64ull << 20;

enum Slot {
    SL_TIN, SL_QIN, SL_TP, SL_QP, SL_QM, SL_KEYS_A, SL_KEYS_B, SL_BCOUNT, SL_OFFS, SL_POS,
    SL_COUNTS, SL_STARTS, SL_HITS_A, SL_HITS_B, SL_QUEUE, SL_PAIRS, SL_BENTRIES, SL_SCHED,
    SL_HSPS, SL_TMP, SL_ECARRY, SL_PUB, SL_BOUNDS, SL_BSLOTS, SL_OFF2, SL_POS2, SL_PLANES, SL_LOW,
    SL_YANCH, SL_YHALF, NSLOT
};

// Small device block: scores, counters and flags of one call.
struct Small {
    int32_t scores[16];
    DevCounters ctr;
    uint32_t status;       // pack / conversion status
    uint32_t queue_len;
    unsigned long long split;
    uint32_t work_next;    // persistent walk: next chunk ticket
    uint32_t warps_done;   // persistent walk: warps out of lane work
    uint32_t queue_take;   // persistent walk: next queue entry to consume
    uint32_t pad0;
    unsigned long long pad[2];
};

int bits_for(long long v) {
    int b = 1;
    while (b < 63 && (1LL << b) <= v) b++;
    return b;
}

}  // namespace

// CUDA-event spans of the stages of one call (SFE_TIME_STAGES).
struct StageTimer {
    struct Span {
        int stage;
        cudaEvent_t a, b;
        unsigned long long l0, l1;
    };
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<Span> spans;
};

struct sfe_ctx {
    int device = 0;
    cudaStream_t own = nullptr;
    cudaStream_t st = nullptr;
    void *buf[NSLOT] = {};
    size_t cap[NSLOT] = {};
    Small *small = nullptr;       // device
    Small *host_small = nullptr;  // pinned mirror
    uint32_t epoch = 0;           // tag of the current call's hand-off queue entries
    unsigned long long batch_hits_hint = 0;  // hits of the last batch (room for the next)
    StageTimer tm;
    unsigned long long launches0 = 0;
    int fail_allocs = 0;  // test hook: allocations still to fail
    sfe_params walk{};    // walk settings of sfe_ungapped_xdrop (sfe_ctx_set_walk)
    bool walk_set = false;
};

struct sfe_index {
    int device = 0;
    long long tlen = 0;
    SeedPattern pat{};
    int transition = 1;
    int codes = 0;                 // input format of the target, reused for queries
    uint32_t *tp_alloc = nullptr;  // packed target with padding
    uint32_t *offs = nullptr;      // 4^weight + 1
    uint32_t *pos = nullptr;       // tlen - span + 1
    uint32_t *ncount = nullptr;    // 4^weight: hits of each key's probe set
    uint32_t *off2 = nullptr;      // merged probe-set lists (optional): 4^weight + 1
    uint32_t *pos2 = nullptr;      //   and (1 + weight) x positions
    int shift = 0;                 // sparse index: CSR over key >> shift ...
    uint16_t *low = nullptr;       //   and each entry's key & (2^shift - 1)
};

namespace {

int ensure(sfe_ctx *c, int slot, size_t bytes, void **out) {
    if (bytes < 256) bytes = 256;
    if (c->cap[slot] < bytes) {
        if (c->fail_allocs > 0) {
            c->fail_allocs--;
            return fail(SFE_ENOMEM, "device allocation failed (injected by the test hook)");
        }
        if (c->buf[slot]) {
            CK(cudaFreeAsync(c->buf[slot], c->st));
            c->buf[slot] = nullptr;
            c->cap[slot] = 0;
        }
        size_t nb = bytes + bytes / 8;
        void *p = nullptr;
        cudaError_t e = cudaMallocAsync(&p, nb, c->st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SFE_ENOMEM, "device allocation of " + std::to_string(nb) + " bytes failed");
        }
        c->buf[slot] = p;
        c->cap[slot] = nb;
    }
    *out = c->buf[slot];
    return SFE_OK;
}

template <typename T>
int ensure_t(sfe_ctx *c, int slot, size_t count, T **out) {
    void *p = nullptr;
    TRY(ensure(c, slot, count * sizeof(T), &p));
    *out = reinterpret_cast<T *>(p);
    return SFE_OK;
}

cudaEvent_t next_event(sfe_ctx *c) {
    StageTimer &t = c->tm;
    if (t.used < t.pool.size()) return t.pool[t.used++];
    if (t.pool.size() >= 8192) return nullptr;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    t.pool.push_back(e);
    t.used++;
    return e;
}

// RAII span: events recorded on the context's stream around one stage.
struct Span {
    sfe_ctx *c;
    int stage;
    cudaEvent_t a = nullptr;
    unsigned long long l0;
    Span(sfe_ctx *ctx, int s) : c(ctx), stage(s), l0(g_launches) {
        if (c->tm.on && (a = next_event(c))) cudaEventRecord(a, c->st);
    }
    ~Span() {
        if (!a) return;
        cudaEvent_t b = next_event(c);
        if (!b) return;
        cudaEventRecord(b, c->st);
        c->tm.spans.push_back({stage, a, b, l0, g_launches});
    }
};

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int parse_pattern(const char *s, SeedPattern *p) {
    if (!s) s = kDefaultPattern;
    int n = (int)strlen(s);
    if (n < 1 || n > MAX_SPAN) return fail(SFE_EINVAL, "seed pattern span must be 1..32");
    memset(p, 0, sizeof(*p));
    p->span = n;
    p->step = 1;
    for (int i = 0; i < n; i++) {
        if (s[i] == '1')
            p->care[p->weight++] = i;
        else if (s[i] != '0')
            return fail(SFE_EINVAL, "seed pattern holds a character other than 0/1");
    }
    if (p->weight < 1 || p->weight > MAX_WEIGHT)
        return fail(SFE_EINVAL, "seed pattern weight must be 1..14");
    return SFE_OK;
}

int check_params(const sfe_params *p) {
    if (!p) return fail(SFE_EINVAL, "params is NULL");
    if (p->xdrop < 0 || p->xdrop >= (1 << 30)) return fail(SFE_EINVAL, "xdrop must be in [0, 2^30)");
    if (p->strands < 1 || p->strands > 3) return fail(SFE_EINVAL, "strands must be 1, 2 or 3");
    if (p->lane_cap < 0) return fail(SFE_EINVAL, "lane_cap must be >= 0");
    if (p->lanes_per_sm < 0) return fail(SFE_EINVAL, "lanes_per_sm must be >= 0");
    if (p->walk_chunk < 0) return fail(SFE_EINVAL, "walk_chunk must be >= 0");
    if (p->walk_mode != SFE_WALK_PERSISTENT && p->walk_mode != SFE_WALK_TWO_LAUNCHES &&
        p->walk_mode != SFE_WALK_SPECULATIVE)
        return fail(SFE_EINVAL, "walk_mode must be SFE_WALK_PERSISTENT, SFE_WALK_TWO_LAUNCHES or "
                                "SFE_WALK_SPECULATIVE");
    if (p->spec_window < 0 || p->spec_window > 32 || (p->spec_window & (p->spec_window - 1)))
        return fail(SFE_EINVAL, "spec_window must be 0 or a power of two up to 32");
    if (p->walk_schedule < SFE_SCHED_NATURAL || p->walk_schedule > SFE_SCHED_RANDOM)
        return fail(SFE_EINVAL, "unknown walk_schedule");
    if (p->walk_schedule != SFE_SCHED_NATURAL && p->walk_mode != SFE_WALK_PERSISTENT)
        return fail(SFE_EINVAL, "a walk_schedule other than natural needs SFE_WALK_PERSISTENT");
    if (p->walk_schedule == SFE_SCHED_PREDICTED && (!p->model || !is_device_ptr(p->model)))
        return fail(SFE_EINVAL, "SFE_SCHED_PREDICTED needs params.model in device memory");
    if (p->ext_log_every < 0 || p->ext_log_cap < 0) return fail(SFE_EINVAL, "bad ext_log settings");
    if (p->ext_log && p->ext_log_every > 0 && !is_device_ptr(p->ext_log))
        return fail(SFE_EINVAL, "ext_log must be device memory");
    if (p->tile_hits < 0) return fail(SFE_EINVAL, "tile_hits must be >= 0");
    if (p->input_codes != 0 && p->input_codes != 1) return fail(SFE_EINVAL, "input_codes must be 0 or 1");
    if (p->step < 0) return fail(SFE_EINVAL, "step must be >= 0");
    for (int i = 0; i < 16; i++)
        if (p->scores[i] < -(1 << 20) || p->scores[i] > (1 << 20))
            return fail(SFE_EINVAL, "scores must lie in [-2^20, 2^20]");
    return SFE_OK;
}

int check_len(long long n, const char *what) {
    if (n < 0 || n > (long long)INT_MAX - 1024)
        return fail(SFE_EINVAL, std::string(what) + " length must be in [0, 2^31 - 1024]");
    return SFE_OK;
}

// A walk packs the diagonal index t - q + (qlen - span) in 31 bits (the hit
// list's walk layout keeps the strand in the top bit of the word), so a
// target and a query walked together stay below 2^31 bases.
int check_pair(long long tlen, long long qlen) {
    if (tlen + qlen > (long long)INT_MAX)
        return fail(SFE_EINVAL, "target and query together must be shorter than 2^31 bases");
    return SFE_OK;
}

int begin(sfe_ctx *c, int flags = 0) {
    if (!c) return fail(SFE_EINVAL, "context is NULL");
    CK(cudaSetDevice(c->device));
    c->tm.on = (flags & SFE_TIME_STAGES) != 0;
    c->tm.used = 0;
    c->tm.spans.clear();
    c->launches0 = g_launches;
    CK(cudaMemsetAsync(c->small, 0, sizeof(Small), c->st));
    return SFE_OK;
}

// Bytes in (host or device) -> device pointer (host data copied to `slot`).
int stage(sfe_ctx *c, int slot, const void *src, size_t bytes, const void **dev) {
    if (bytes == 0 || is_device_ptr(src)) {
        *dev = src;
        return SFE_OK;
    }
    if (!src) return fail(SFE_EINVAL, "input pointer is NULL");
    void *d = nullptr;
    TRY(ensure(c, slot, bytes, &d));
    CK(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, c->st));
    *dev = d;
    return SFE_OK;
}

size_t packed_words(long long n) { return (size_t)((n + 15) / 16) + 2 * SEQ_PAD; }

// Pack `n` bases from `src` (device) into a padded buffer; returns base-0 pointer.
int pack_into(sfe_ctx *c, const uint8_t *src, long long n, int codes, uint32_t *alloc,
              uint32_t **base0) {
    *base0 = alloc + SEQ_PAD;
    CK(launch_pack(src, n, codes, *base0, &c->small->status, c->st));
    return SFE_OK;
}

int pack_slot(sfe_ctx *c, int slot, const uint8_t *src, long long n, int codes, uint32_t **base0) {
    uint32_t *a = nullptr;
    TRY(ensure_t(c, slot, packed_words(n), &a));
    return pack_into(c, src, n, codes, a, base0);
}

int rc_slot(sfe_ctx *c, int slot, const uint32_t *fwd, long long n, uint32_t **base0) {
    uint32_t *a = nullptr;
    TRY(ensure_t(c, slot, packed_words(n), &a));
    *base0 = a + SEQ_PAD;
    CK(launch_revcomp(fwd, n, *base0, c->st));
    return SFE_OK;
}

int sync_small(sfe_ctx *c) {
    CK(cudaMemcpyAsync(c->host_small, c->small, sizeof(Small), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return SFE_OK;
}

int check_status(uint32_t st) {
    if (st & ST_BAD_SYMBOL) return fail(SFE_EINVAL, "sequence holds a symbol outside ACGTacgt");
    if (st & ST_BAD_HIT) return fail(SFE_EINVAL, "a hit's seed span leaves the sequences");
    if (st & ST_SCORE_OVERFLOW) return fail(SFE_EOVERFLOW, "an HSP score left the int32 range");
    if (st & ST_TIMEOUT) return fail(SFE_ETIMEOUT, "a bounded device wait ran out");
    return SFE_OK;
}

struct IndexView {
    const uint32_t *T;
    long long tlen;
    SeedPattern pat;
    int transition;
    const uint32_t *offs;
    const uint32_t *pos;
    const uint32_t *ncount;
    const uint32_t *off2, *pos2;  // merged probe-set lists, or null
    int shift;                    // sparse index (low != null): buckets are key >> shift
    const uint16_t *low;
};

HitParams hit_params(const IndexView &v, long long qlen) {
    HitParams hp;
    hp.pat = v.pat;
    hp.transition = v.transition;
    hp.qlen = qlen;
    hp.qoff = qlen - v.pat.span;
    hp.shift = v.shift;
    hp.low = v.low;
    return hp;
}

// Entries of the merged probe-set lists: every position is read by the probe
// sets of 1 + weight keys (the relation "is a probe of" is symmetric). They
// are kept while they fit u32 offsets and a memory budget.
long long merged_entries(const SeedPattern &pat, int transition, long long tlen) {
    return (transition ? pat.weight + 1 : 1) * indexed_positions(pat, tlen);
}
// The per-key tables (probe-set sizes, merged lists) are built over all
// 4^weight keys; they pay only while the target fills them: with at most one
// indexed position per four keys (a weight-14 seed on a 10 Mb target) the
// count and write passes probe the CSR offsets of the 1 + weight keys instead.
bool dense_tables(const SeedPattern &pat, long long tlen) {
    return (1LL << (2 * pat.weight)) <= 4 * indexed_positions(pat, tlen);
}
// Sparse index: buckets are the top 2 * weight - shift key bits, about one
// indexed position per bucket (and at least 2^(2 * weight - 16) buckets, so
// the remaining bits fit the 16-bit low column). 0 for a dense index.
int index_shift(const SeedPattern &pat, long long tlen, bool force_dense = false) {
    if (force_dense || dense_tables(pat, tlen)) return 0;
    int cb = 1;
    while (cb < 2 * pat.weight && (1LL << cb) < indexed_positions(pat, tlen)) cb++;
    cb = std::max(cb, 2 * pat.weight - 16);
    return 2 * pat.weight - cb;
}
bool use_merged(const SeedPattern &pat, int transition, long long tlen, int shift) {
    const long long m = merged_entries(pat, transition, tlen);
    return shift == 0 && m < (1LL << 32) - 1 && m * 4 <= (16LL << 30);
}

// Spaced keys -> stable radix sort -> CSR (offsets, positions).
// ncount (4^weight entries, may be the arena's bucket counts once the scan is
// done) receives the hits of every key's probe set under `transition`.
// off2 / pos2 (optional) receive the merged probe-set lists.
int build_index(sfe_ctx *c, const uint32_t *T, long long tlen, const SeedPattern &pat,
                int transition, int shift, uint32_t *offs, uint32_t *pos, uint32_t **ncount_io,
                uint32_t *off2 = nullptr, uint32_t *pos2 = nullptr, uint16_t *low = nullptr) {
    const long long npos = indexed_positions(pat, tlen);
    const long long nbuckets = 1LL << (2 * pat.weight - shift);
    uint32_t *counts = nullptr;
    TRY(ensure_t(c, SL_BCOUNT, (size_t)nbuckets, &counts));
    CK(cudaMemsetAsync(counts, 0, (size_t)nbuckets * 4, c->st));
    void *tmp = nullptr;
    TRY(ensure(c, SL_TMP, std::max(radix_sort_temp_bytes(npos), scan_temp_bytes(nbuckets)), &tmp));
    if (npos > 0) {
        uint64_t *ka = nullptr, *kb = nullptr;
        TRY(ensure_t(c, SL_KEYS_A, (size_t)npos, &ka));
        TRY(ensure_t(c, SL_KEYS_B, (size_t)npos, &kb));
        CK(launch_seed_keys(T, tlen, pat, ka, c->st));
        bool in_b = false;
        CK(radix_sort(ka, kb, nullptr, nullptr, npos, 32, 32 + 2 * pat.weight, tmp, &in_b, &c->small->status, c->st));
        CK(launch_csr_counts(in_b ? kb : ka, npos, counts, pos, shift, shift ? low : nullptr,
                             c->st));
    }
    CK(scan_u32_to_u32(counts, offs, nbuckets, tmp, c->st));
    if (shift) {  // sparse: the hit passes probe the buckets
        *ncount_io = nullptr;
        return SFE_OK;
    }
    if (!*ncount_io) *ncount_io = counts;  // the per-key counts are no longer needed
    CK(launch_neighbor_counts(offs, pat, transition, *ncount_io, c->st));
    if (off2 && pos2) {
        CK(scan_u32_to_u32(*ncount_io, off2, nbuckets, tmp, c->st));
        CK(launch_merged_fill(offs, pos, pat, transition, off2, pos2, c->st));
    }
    return SFE_OK;
}

// Count pass + exclusive scan of one strand; returns the total on the host.
int count_hits(sfe_ctx *c, const IndexView &ix, const uint32_t *Qs, long long qlen,
               unsigned long long **starts_out, long long *nq_out, unsigned long long *total) {
    *total = 0;
    const long long nq = qlen - ix.pat.span + 1;
    *nq_out = nq;
    if (nq <= 0 || ix.tlen < ix.pat.span) {
        *nq_out = 0;
        return SFE_OK;
    }
    const HitParams hp = hit_params(ix, qlen);
    uint32_t *counts = nullptr;
    unsigned long long *starts = nullptr;
    void *tmp = nullptr;
    TRY(ensure_t(c, SL_COUNTS, (size_t)nq, &counts));
    TRY(ensure_t(c, SL_STARTS, (size_t)nq + 1, &starts));
    TRY(ensure(c, SL_TMP, scan_temp_bytes(nq), &tmp));
    CK(launch_hit_count(Qs, hp, ix.offs, ix.ncount, 0, nq, counts, c->st));
    CK(scan_u32_to_u64(counts, starts, nq, tmp, c->st));
    CK(cudaMemcpyAsync(total, starts + nq, 8, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    *starts_out = starts;
    return SFE_OK;
}

__global__ void tile_bounds_kernel(const unsigned long long *starts, long long nq,
                                   unsigned long long per, long long ntiles, long long *bounds,
                                   unsigned long long *bstarts) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k > ntiles) return;
    long long b;
    if (k == 0) {
        b = 0;
    } else if (k == ntiles) {
        b = nq;
    } else {
        unsigned long long target = per * (unsigned long long)k;
        long long lo = 0, hi = nq;  // first q with starts[q] >= target
        while (lo < hi) {
            long long mid = (lo + hi) / 2;
            if (starts[mid] < target)
                lo = mid + 1;
            else
                hi = mid;
        }
        b = lo;
    }
    bounds[k] = b;
    bstarts[k] = starts[b];
}

__global__ void strand_split_kernel(const uint64_t *keys, long long n, unsigned long long *split) {
    long long lo = 0, hi = n;  // first index with bit 63 set
    while (lo < hi) {
        long long mid = (lo + hi) / 2;
        if ((keys[mid] >> 63) == 0)
            lo = mid + 1;
        else
            hi = mid;
    }
    *split = (unsigned long long)lo;
}

struct WalkSetup {
    const uint32_t *T;
    long long tlen;
    const uint32_t *Qs;
    long long qlen;
    int strand;
    int span;
    const sfe_params *p;
    int32_t *Ecarry;
    Hsp *hsps;
    unsigned long long hsp_cap;
    const uint32_t *planes[2] = {nullptr, nullptr};  // cell planes of T and of Qs
};

// The lane and warp tiers over hits sorted by (diagonal word, t), in one
// persistent launch or as two launches (params->walk_mode).
// `sm` is the counter block (the context's by default) and `sched_tmp` the
// schedule's scratch (taken from the arena by default); both are given by a
// batch plan, whose captured graph must own every buffer it touches.
int walk_tiers(sfe_ctx *c, const uint64_t *hits, long long n, WalkParams &wp, uint4 *queue,
               unsigned long long qcap, const sfe_params *p, Small *sm = nullptr,
               void *sched_tmp = nullptr) {
    if (!sm) sm = c->small;
    if (p->ext_log && p->ext_log_every > 0) {
        wp.elog = p->ext_log;
        wp.elog_cap = (unsigned long long)std::max<int64_t>(0, p->ext_log_cap);
        wp.elog_every = (uint32_t)p->ext_log_every;
    }
    wp.queue = queue;
    wp.queue_cap = qcap;
    wp.queue_len = &sm->queue_len;
    CK(cudaMemsetAsync(&sm->queue_len, 0, 4, c->st));
    if (p->walk_mode == SFE_WALK_SPECULATIVE) {
        Span sp(c, SFE_STAGE_WALK_WARPS);
        wp.work_next = &sm->work_next;
        wp.chunk = p->walk_chunk > 0 ? (uint32_t)p->walk_chunk : walk_auto_chunk(n);
        CK(cudaMemsetAsync(&sm->work_next, 0, 4, c->st));
        CK(launch_walk_speculative(hits, n, wp, p->spec_window > 0 ? p->spec_window : 8, c->st));
        return SFE_OK;
    }
    if (p->walk_mode == SFE_WALK_TWO_LAUNCHES) {
        {
            Span sp(c, SFE_STAGE_WALK_LANES);
            CK(launch_walk_lanes(hits, n, wp, p->lanes_per_sm, c->st));
        }
        Span sp(c, SFE_STAGE_WALK_WARPS);
        CK(launch_walk_warps(hits, n, wp, 0, c->st));
        return SFE_OK;
    }
    if (++c->epoch == 0) c->epoch = 1;
    wp.epoch = c->epoch;
    wp.work_next = &sm->work_next;
    wp.warps_done = &sm->warps_done;
    wp.queue_take = &sm->queue_take;
    wp.chunk = p->walk_chunk > 0 ? (uint32_t)p->walk_chunk : walk_auto_chunk(n);
    wp.order = nullptr;
    wp.spin_limit = p->wait_limit > 0 ? p->wait_limit : (1LL << 20);
    wp.phantom = (p->test_hooks & SFE_TEST_UNPUBLISHED_QUEUE_ENTRY) ? 1 : 0;
    if (p->walk_schedule != SFE_SCHED_NATURAL) {
        Span sp(c, SFE_STAGE_SCHEDULE);
        void *tmp = sched_tmp;
        if (!tmp) TRY(ensure(c, SL_SCHED, walk_schedule_temp_bytes(n, wp.chunk), &tmp));
        uint32_t *order = nullptr;
        CK(launch_walk_schedule(hits, n, wp, p->walk_schedule, p->model, tmp, &order,
                                &sm->status, c->st));
        wp.order = order;
    }
    {
        Span sp(c, SFE_STAGE_WALK_LANES);
        CK(cudaMemsetAsync(&sm->work_next, 0, 12, c->st));
        CK(cudaMemsetAsync(queue, 0, (size_t)qcap * sizeof(uint4), c->st));
        CK(launch_walk_persistent(hits, n, wp, c->st));
    }
    // entries whose consumers gave up waiting (the persistent grid does not
    // fit on the device at once, e.g. next to another kernel) are walked here,
    // after every producer has finished; normally nothing is left
    Span sp(c, SFE_STAGE_WALK_WARPS);
    WalkParams fu = wp;
    fu.deferred_only = 1;
    CK(launch_walk_warps(hits, n, fu, 2 * device_sms() * (BLOCK / 32), c->st));
    return SFE_OK;
}

// Lane and warp walks of hits sorted by (diagonal, t).
int walk_sorted(sfe_ctx *c, const uint64_t *hits, long long n, const WalkSetup &ws) {
    if (n <= 0) return SFE_OK;
    uint4 *queue = nullptr;
    const unsigned long long qcap = std::min<unsigned long long>((unsigned long long)n, kQueueMax);
    TRY(ensure_t(c, SL_QUEUE, (size_t)qcap, &queue));
    WalkParams wp{};
    wp.T = ws.T;
    wp.Q = ws.Qs;
    wp.TN = ws.planes[0];
    wp.QN = ws.planes[1];
    wp.tlen = ws.tlen;
    wp.qlen = ws.qlen;
    wp.span = ws.span;
    wp.strand = ws.strand;
    wp.xdrop = ws.p->xdrop;
    wp.thresh = ws.p->hsp_thresh;
    wp.flags = ws.p->flags;
    wp.lane_cap = ws.p->lane_cap > 0 ? ws.p->lane_cap : DEFAULT_LANE_CAP;
    wp.qoff = ws.qlen - ws.span;
    wp.scores = c->small->scores;
    wp.Ecarry = ws.Ecarry;
    wp.hsps = ws.hsps;
    wp.hsp_cap = ws.hsp_cap;
    wp.ctr = &c->small->ctr;
    return walk_tiers(c, hits, n, wp, queue, qcap, ws.p);
}

// Sort the HSPs found and copy them out; sets *nhsps (SFE_EOVERFLOW if > cap).
int finish_hsps(sfe_ctx *c, Hsp *dev, unsigned long long found, long long tlen, long long qlen,
                sfe_hsp *out, int64_t cap, int64_t *nhsps) {
    *nhsps = (int64_t)found;
    if ((long long)found > cap) return fail(SFE_EOVERFLOW, "HSP buffer too small");
    if (found == 0) return SFE_OK;
    void *tmp = nullptr;
    TRY(ensure(c, SL_TMP, hsp_sort_temp_bytes((long long)found), &tmp));
    CK(hsp_sort(dev, (long long)found, bits_for(tlen), bits_for(qlen), tmp, &c->small->status, c->st));
    const bool dev_out = is_device_ptr(out);
    CK(cudaMemcpyAsync(out, dev, found * sizeof(Hsp),
                       dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return SFE_OK;
}

void fill_stats(const Small &s, sfe_stats *st, long long hits, long long tiles) {
    if (!st) return;
    memset(st, 0, sizeof(*st));
    st->hits = hits;
    st->extended = (int64_t)s.ctr.extended;
    st->cells = (int64_t)s.ctr.cells;
    st->hsps = (int64_t)s.ctr.hsps;
    st->lane_tasks = (int64_t)s.ctr.lane_tasks;
    st->warp_tasks = (int64_t)s.ctr.warp_tasks;
    st->warp_cells = (int64_t)s.ctr.warp_cells;
    st->ext_logged = (int64_t)s.ctr.ext_logged;
    st->shadow_cells = (int64_t)s.ctr.shadow;
    st->deferred_tasks = (int64_t)s.ctr.deferred;
    st->tiles = tiles;
}

// Stage times and launch counts (after the stream has been synchronised).
void add_timings(sfe_ctx *c, sfe_stats *st) {
    if (!st) return;
    st->launches = (int64_t)(g_launches - c->launches0);
    for (const auto &sp : c->tm.spans) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, sp.a, sp.b) == cudaSuccess) st->stage_ms[sp.stage] += ms;
        else cudaGetLastError();
        st->stage_launches[sp.stage] += (int64_t)(sp.l1 - sp.l0);
    }
    c->tm.spans.clear();
}

int upload_scores(sfe_ctx *c, const int32_t *scores) {
    CK(cudaMemcpyAsync(c->small->scores, scores, 64, cudaMemcpyHostToDevice, c->st));
    return SFE_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" {

int sfe_params_default(sfe_params *p) {
    if (!p) return fail(SFE_EINVAL, "params is NULL");
    memset(p, 0, sizeof(*p));
    p->seed_pattern = kDefaultPattern;
    p->transition = 1;
    p->strands = 3;
    memcpy(p->scores, kHoxd70, sizeof(kHoxd70));
    p->xdrop = 910;
    p->hsp_thresh = 3000;
    // measured on the 10 Mb and 100 Mb pairs: the persistent walk with chunks
    // of 64 hits is 0.5-1.3% faster than two launches with fixed hit ranges;
    // smaller inputs get smaller chunks (walk_chunk 0: from the hit count)
    p->walk_mode = SFE_WALK_PERSISTENT;
    p->walk_chunk = 0;
    return SFE_OK;
}

const char *sfe_strerror(int code) {
    switch (code) {
    case SFE_OK: return "ok";
    case SFE_EINVAL: return "invalid argument";
    case SFE_ENOMEM: return "out of device memory";
    case SFE_ECUDA: return "CUDA error";
    case SFE_ETIMEOUT: return "bounded device wait ran out";
    case SFE_EOVERFLOW: return "output capacity or int32 range exceeded";
    case SFE_ELIMIT: return "input larger than the fixed scratch of the allocation-free call";
    default: return "unknown error";
    }
}

const char *sfe_last_error(void) { return g_err.c_str(); }

int sfe_ctx_create(int device, sfe_ctx **out) {
    if (!out) return fail(SFE_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(SFE_EINVAL, "no such CUDA device");
    CK(cudaSetDevice(device));
    sfe_ctx *c = new sfe_ctx();
    c->device = device;
    cudaError_t e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&c->small, sizeof(Small));
    if (e == cudaSuccess) e = cudaMallocHost(&c->host_small, sizeof(Small));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (c->small) cudaFree(c->small);
        if (c->own) cudaStreamDestroy(c->own);
        delete c;
        return fail(SFE_ECUDA, std::string("context setup: ") + cudaGetErrorString(e));
    }
    c->st = c->own;
    *out = c;
    return SFE_OK;
}

int sfe_test_radix_sort(sfe_ctx *c, uint64_t *keys, int64_t n, int32_t lo, int32_t hi,
                        int32_t device_count) {
    TRY(begin(c));
    if (n < 0 || n >= (1LL << 32) || lo < 0 || hi > 64 || lo >= hi)
        return fail(SFE_EINVAL, "bad count or bit range");
    if (n > 0 && !is_device_ptr(keys)) return fail(SFE_EINVAL, "keys must be device memory");
    if (n <= 1) return SFE_OK;
    uint64_t *other = nullptr;
    void *tmp = nullptr;
    unsigned long long *nd = nullptr;
    TRY(ensure_t(c, SL_HITS_B, (size_t)n, &other));
    TRY(ensure(c, SL_TMP, radix_sort_temp_bytes(n), &tmp));
    if (device_count) {
        TRY(ensure_t(c, SL_BOUNDS, 1, &nd));
        const unsigned long long hn = (unsigned long long)n;
        CK(cudaMemcpyAsync(nd, &hn, 8, cudaMemcpyHostToDevice, c->st));
    }
    bool in_b = false;
    CK(radix_sort_dev(keys, other, nullptr, nullptr, n, nd, lo, hi, tmp, &in_b,
                      &c->small->status, c->st));
    if (in_b)
        CK(cudaMemcpyAsync(keys, other, (size_t)n * 8, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    return SFE_OK;
}

int sfe_ctx_set_walk(sfe_ctx *c, const sfe_params *params) {
    if (!c) return fail(SFE_EINVAL, "context is NULL");
    if (!params) {
        c->walk_set = false;
        return SFE_OK;
    }
    sfe_params p;
    sfe_params_default(&p);
    p.walk_mode = params->walk_mode;
    p.lane_cap = params->lane_cap;
    p.walk_chunk = params->walk_chunk;
    p.spec_window = params->spec_window;
    p.flags = params->flags & SFE_TIME_STAGES;
    TRY(check_params(&p));
    c->walk = p;
    c->walk_set = true;
    return SFE_OK;
}

int sfe_ctx_fail_next_allocs(sfe_ctx *c, int32_t n) {
    if (!c || n < 0) return fail(SFE_EINVAL, "bad context or count");
    c->fail_allocs = n;
    return SFE_OK;
}

int sfe_ctx_set_stream(sfe_ctx *c, void *stream) {
    if (!c) return fail(SFE_EINVAL, "context is NULL");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->st));
    c->st = stream ? reinterpret_cast<cudaStream_t>(stream) : c->own;
    return SFE_OK;
}

void sfe_ctx_destroy(sfe_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->st);
    for (cudaEvent_t e : c->tm.pool) cudaEventDestroy(e);
    for (int i = 0; i < NSLOT; i++)
        if (c->buf[i]) cudaFreeAsync(c->buf[i], c->st);
    cudaStreamSynchronize(c->st);
    if (c->small) cudaFree(c->small);
    if (c->host_small) cudaFreeHost(c->host_small);
    if (c->own) cudaStreamDestroy(c->own);
    delete c;
}

int sfe_index_build(sfe_ctx *c, const uint8_t *target, int64_t tlen, const sfe_params *params,
                    sfe_index **out) {
    if (!out) return fail(SFE_EINVAL, "out is NULL");
    *out = nullptr;
    TRY(check_len(tlen, "target"));
    SeedPattern pat;
    TRY(parse_pattern(params ? params->seed_pattern : nullptr, &pat));
    if (params && params->step < 0) return fail(SFE_EINVAL, "step must be >= 0");
    pat.step = params && params->step > 1 ? params->step : 1;
    const int codes = params ? params->input_codes : 0;
    TRY(begin(c));
    const void *tdev = nullptr;
    TRY(stage(c, SL_TIN, target, (size_t)tlen, &tdev));
    sfe_index *ix = new sfe_index();
    ix->device = c->device;
    ix->tlen = tlen;
    ix->pat = pat;
    ix->transition = params ? params->transition : 1;
    ix->codes = codes;
    const long long npos = indexed_positions(pat, tlen);
    ix->shift = index_shift(pat, tlen, params && (params->test_hooks & SFE_TEST_DENSE_INDEX));
    const long long nbuckets = 1LL << (2 * pat.weight - ix->shift);
    cudaError_t e = cudaMalloc(&ix->tp_alloc, packed_words(tlen) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&ix->offs, (size_t)(nbuckets + 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&ix->pos, (size_t)std::max(1LL, npos) * 4);
    if (e == cudaSuccess && ix->shift)
        e = cudaMalloc(&ix->low, (size_t)std::max(1LL, npos) * 2);
    if (e == cudaSuccess && !ix->shift) e = cudaMalloc(&ix->ncount, (size_t)nbuckets * 4);
    if (e == cudaSuccess && use_merged(pat, ix->transition, tlen, ix->shift)) {
        e = cudaMalloc(&ix->off2, (size_t)(nbuckets + 1) * 4);
        if (e == cudaSuccess)
            e = cudaMalloc(&ix->pos2,
                           (size_t)std::max(1LL, merged_entries(pat, ix->transition, tlen)) * 4);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        sfe_index_free(ix);
        return fail(SFE_ENOMEM, "index allocation failed");
    }
    uint32_t *T = nullptr;
    int r = pack_into(c, reinterpret_cast<const uint8_t *>(tdev), tlen, codes, ix->tp_alloc, &T);
    if (r == SFE_OK)
        r = build_index(c, T, tlen, pat, ix->transition, ix->shift, ix->offs, ix->pos,
                        &ix->ncount, ix->off2, ix->pos2, ix->low);
    if (r == SFE_OK) r = sync_small(c);
    if (r == SFE_OK) r = check_status(c->host_small->status);
    if (r != SFE_OK) {
        sfe_index_free(ix);
        return r;
    }
    *out = ix;
    return SFE_OK;
}

void sfe_index_free(sfe_index *ix) {
    if (!ix) return;
    cudaSetDevice(ix->device);
    if (ix->tp_alloc) cudaFree(ix->tp_alloc);
    if (ix->offs) cudaFree(ix->offs);
    if (ix->pos) cudaFree(ix->pos);
    if (ix->ncount) cudaFree(ix->ncount);
    if (ix->off2) cudaFree(ix->off2);
    if (ix->pos2) cudaFree(ix->pos2);
    if (ix->low) cudaFree(ix->low);
    delete ix;
}

static IndexView view_of(const sfe_index *ix) {
    IndexView v;
    v.T = ix->tp_alloc + SEQ_PAD;
    v.tlen = ix->tlen;
    v.pat = ix->pat;
    v.transition = ix->transition;
    v.offs = ix->offs;
    v.pos = ix->pos;
    v.ncount = ix->ncount;
    v.off2 = ix->off2;
    v.pos2 = ix->pos2;
    v.shift = ix->shift;
    v.low = ix->low;
    return v;
}

int sfe_seed_hits(sfe_ctx *c, const sfe_index *ix, const uint8_t *query, int64_t qlen,
                  int32_t strands, sfe_hit *hits, int64_t cap, int64_t *nhits) {
    if (!ix || !nhits) return fail(SFE_EINVAL, "index or nhits is NULL");
    if (strands < 1 || strands > 3) return fail(SFE_EINVAL, "strands must be 1, 2 or 3");
    TRY(check_len(qlen, "query"));
    TRY(check_pair(ix->tlen, qlen));
    TRY(begin(c));
    const IndexView v = view_of(ix);
    const void *qdev = nullptr;
    TRY(stage(c, SL_QIN, query, (size_t)qlen, &qdev));
    uint32_t *Qp = nullptr, *Qm = nullptr;
    TRY(pack_slot(c, SL_QP, reinterpret_cast<const uint8_t *>(qdev), qlen, ix->codes, &Qp));
    TRY(rc_slot(c, SL_QM, Qp, qlen, &Qm));
    TRY(sync_small(c));
    TRY(check_status(c->host_small->status));
    unsigned long long tot[2] = {0, 0};
    long long nq = 0;
    for (int s = 0; s < 2; s++) {
        if (!(strands & (1 << s))) continue;
        unsigned long long *starts = nullptr;
        TRY(count_hits(c, v, s ? Qm : Qp, qlen, &starts, &nq, &tot[s]));
    }
    const unsigned long long need = tot[0] + tot[1];
    *nhits = (int64_t)need;
    if ((long long)need > cap) return fail(SFE_EOVERFLOW, "hit buffer too small");
    if (need == 0) return SFE_OK;
    const bool dev_out = is_device_ptr(hits);
    sfe_hit *dst = hits;
    if (!dev_out) TRY(ensure_t(c, SL_PUB, (size_t)need, &dst));
    unsigned long long at = 0;
    const int DB = bits_for(ix->tlen + qlen - 2LL * v.pat.span);
    for (int s = 0; s < 2; s++) {
        if (!(strands & (1 << s)) || tot[s] == 0) continue;
        unsigned long long *starts = nullptr;
        unsigned long long t2 = 0;
        TRY(count_hits(c, v, s ? Qm : Qp, qlen, &starts, &nq, &t2));
        uint64_t *ha = nullptr, *hb = nullptr;
        void *tmp = nullptr;
        TRY(ensure_t(c, SL_HITS_A, (size_t)t2, &ha));
        TRY(ensure_t(c, SL_HITS_B, (size_t)t2, &hb));
        TRY(ensure(c, SL_TMP, radix_sort_temp_bytes((long long)t2), &tmp));
        const HitParams hp = hit_params(v, qlen);
        CK(launch_hit_write(s ? Qm : Qp, hp, v.offs, v.pos, v.off2, v.pos2, 0, nq, starts, 0, t2, ha,
                            c->st));
        bool in_b = false;
        CK(radix_sort(ha, hb, nullptr, nullptr, (long long)t2, 32, 32 + DB, tmp, &in_b, &c->small->status, c->st));
        CK(launch_hits_to_public(in_b ? hb : ha, (long long)t2, s, hp.qoff, dst + at, c->st));
        at += t2;
    }
    if (!dev_out)
        CK(cudaMemcpyAsync(hits, dst, need * sizeof(sfe_hit), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return SFE_OK;
}

int sfe_ungapped_xdrop(sfe_ctx *c, const sfe_index *ix, const uint8_t *query, int64_t qlen,
                       const sfe_hit *hits, int64_t nhits, const int32_t scores[16], int32_t X,
                       int32_t hsp_thresh, sfe_hsp *hsps, int64_t cap, int64_t *nhsps,
                       sfe_stats *stats) {
    if (!ix || !nhsps || !scores) return fail(SFE_EINVAL, "index, scores or nhsps is NULL");
    if (nhits < 0 || nhits >= (1LL << 32)) return fail(SFE_EINVAL, "nhits out of range");
    TRY(check_len(qlen, "query"));
    TRY(check_pair(ix->tlen, qlen));
    if (!c) return fail(SFE_EINVAL, "context is NULL");
    sfe_params p;
    sfe_params_default(&p);
    if (c->walk_set) {
        p.walk_mode = c->walk.walk_mode;
        p.lane_cap = c->walk.lane_cap;
        p.walk_chunk = c->walk.walk_chunk;
        p.spec_window = c->walk.spec_window;
        p.flags = c->walk.flags;
    }
    memcpy(p.scores, scores, 64);
    p.xdrop = X;
    p.hsp_thresh = hsp_thresh;
    TRY(check_params(&p));
    TRY(begin(c, p.flags));
    const IndexView v = view_of(ix);
    const int span = v.pat.span;
    TRY(upload_scores(c, p.scores));
    const void *qdev = nullptr, *hdev = nullptr;
    TRY(stage(c, SL_QIN, query, (size_t)qlen, &qdev));
    TRY(stage(c, SL_PUB, hits, (size_t)nhits * sizeof(sfe_hit), &hdev));
    uint32_t *Qp = nullptr, *Qm = nullptr;
    TRY(pack_slot(c, SL_QP, reinterpret_cast<const uint8_t *>(qdev), qlen, ix->codes, &Qp));
    TRY(rc_slot(c, SL_QM, Qp, qlen, &Qm));
    uint64_t *ha = nullptr, *hb = nullptr;
    void *tmp = nullptr;
    TRY(ensure_t(c, SL_HITS_A, (size_t)std::max<int64_t>(1, nhits), &ha));
    TRY(ensure_t(c, SL_HITS_B, (size_t)std::max<int64_t>(1, nhits), &hb));
    TRY(ensure(c, SL_TMP, radix_sort_temp_bytes(nhits), &tmp));
    CK(launch_public_to_walk(reinterpret_cast<const sfe_hit *>(hdev), nhits, v.tlen, qlen, span, ha,
                             &c->small->status, c->st));
    TRY(sync_small(c));
    TRY(check_status(c->host_small->status));
    // (strand, diagonal, t): three stable passes, least significant first
    const int TB = bits_for(v.tlen);
    const int DB = bits_for(v.tlen + qlen);
    uint64_t *cur = ha, *oth = hb;
    bool in_b = false;
    CK(radix_sort(cur, oth, nullptr, nullptr, nhits, 0, TB, tmp, &in_b, &c->small->status, c->st));
    if (in_b) std::swap(cur, oth);
    CK(radix_sort(cur, oth, nullptr, nullptr, nhits, 32, 32 + DB, tmp, &in_b, &c->small->status, c->st));
    if (in_b) std::swap(cur, oth);
    CK(radix_sort(cur, oth, nullptr, nullptr, nhits, 63, 64, tmp, &in_b, &c->small->status, c->st));
    if (in_b) std::swap(cur, oth);
    if (nhits > 0) {
        g_launches++;
        strand_split_kernel<<<1, 1, 0, c->st>>>(cur, nhits, &c->small->split);
    }
    CK(cudaGetLastError());
    TRY(sync_small(c));
    const long long split = nhits > 0 ? (long long)c->host_small->split : 0;
    Hsp *hd = nullptr;
    unsigned long long hcap = std::max<unsigned long long>(1ull << 16, (unsigned long long)cap);
    for (int attempt = 0; attempt < 2; attempt++) {
        TRY(ensure_t(c, SL_HSPS, (size_t)hcap, &hd));
        CK(cudaMemsetAsync(&c->small->ctr, 0, sizeof(DevCounters), c->st));
        for (int s = 0; s < 2; s++) {
            const long long b = s ? split : 0, e = s ? nhits : split;
            WalkSetup ws{v.T, v.tlen, s ? Qm : Qp, qlen, s, span, &p, nullptr, hd, hcap};
            TRY(walk_sorted(c, cur + b, e - b, ws));
        }
        TRY(sync_small(c));
        if (c->host_small->ctr.hsps <= hcap) break;
        hcap = c->host_small->ctr.hsps;
    }
    Small sm = *c->host_small;
    TRY(check_status(sm.ctr.status));
    fill_stats(sm, stats, nhits, 1);
    int r = finish_hsps(c, hd, sm.ctr.hsps, v.tlen, qlen, hsps, cap, nhsps);
    add_timings(c, stats);
    return r;
}

int sfe_run(sfe_ctx *c, const uint8_t *target, int64_t tlen, const uint8_t *query, int64_t qlen,
            const sfe_params *params, sfe_hsp *hsps, int64_t cap, int64_t *nhsps,
            sfe_stats *stats) {
    if (!nhsps) return fail(SFE_EINVAL, "nhsps is NULL");
    TRY(check_params(params));
    TRY(check_len(tlen, "target"));
    TRY(check_len(qlen, "query"));
    TRY(check_pair(tlen, qlen));
    SeedPattern pat;
    TRY(parse_pattern(params->seed_pattern, &pat));
    pat.step = params->step > 1 ? params->step : 1;
    TRY(begin(c, params->flags));
    TRY(upload_scores(c, params->scores));
    uint32_t *Tp = nullptr, *Qp = nullptr, *Qm = nullptr;
    {
        Span sp(c, SFE_STAGE_PACK);
        const void *tdev = nullptr, *qdev = nullptr;
        TRY(stage(c, SL_TIN, target, (size_t)tlen, &tdev));
        TRY(stage(c, SL_QIN, query, (size_t)qlen, &qdev));
        TRY(pack_slot(c, SL_TP, reinterpret_cast<const uint8_t *>(tdev), tlen, params->input_codes,
                      &Tp));
        TRY(pack_slot(c, SL_QP, reinterpret_cast<const uint8_t *>(qdev), qlen, params->input_codes,
                      &Qp));
        if (params->strands & 2) TRY(rc_slot(c, SL_QM, Qp, qlen, &Qm));
    }
    // cell planes of T and of each query strand for the lane windows, when
    // they fit well inside L2 (the lanes read them at random positions)
    const uint32_t *planes[2][2] = {};
    {
        const size_t tw = plane_words(tlen), qw = plane_words(qlen);
        const size_t words = tw + 2 * qw;
        if (!(params->flags & SFE_NO_CELL_PLANES) && words * 4 <= kPlanesMaxBytes) {
            Span sp(c, SFE_STAGE_PACK);
            uint32_t *pl = nullptr;
            TRY(ensure_t(c, SL_PLANES, words, &pl));
            uint32_t *tn = pl + PLANE_PAD;
            CK(launch_plane(Tp, tlen, 2, tn, c->st));
            for (int s = 0; s < 2; s++) {
                if (!(params->strands & (1 << s))) continue;
                uint32_t *qn = pl + tw + s * qw + PLANE_PAD;
                CK(launch_plane(s ? Qm : Qp, qlen, 0, qn, c->st));
                planes[s][0] = tn;
                planes[s][1] = qn;
            }
        }
    }
    const long long npos = indexed_positions(pat, tlen);
    const int shift = index_shift(pat, tlen, (params->test_hooks & SFE_TEST_DENSE_INDEX) != 0);
    uint32_t *offs = nullptr, *pos = nullptr;
    uint16_t *low = nullptr;
    TRY(ensure_t(c, SL_OFFS, (size_t)(1LL << (2 * pat.weight - shift)) + 1, &offs));
    TRY(ensure_t(c, SL_POS, (size_t)std::max(1LL, npos), &pos));
    if (shift) TRY(ensure_t(c, SL_LOW, (size_t)std::max(1LL, npos), &low));
    uint32_t *ncount = nullptr, *off2 = nullptr, *pos2 = nullptr;
    if (use_merged(pat, params->transition, tlen, shift)) {
        TRY(ensure_t(c, SL_OFF2, (size_t)(1LL << (2 * pat.weight)) + 1, &off2));
        TRY(ensure_t(c, SL_POS2,
                     (size_t)std::max(1LL, merged_entries(pat, params->transition, tlen)), &pos2));
    }
    {
        Span sp(c, SFE_STAGE_INDEX);
        TRY(build_index(c, Tp, tlen, pat, params->transition, shift, offs, pos, &ncount, off2,
                        pos2, low));
    }
    IndexView v{Tp, tlen, pat, params->transition, offs, pos, ncount, off2, pos2, shift, low};

    const long long tile_hits = params->tile_hits > 0 ? params->tile_hits : kDefaultTileHits;
    const int DB = bits_for(tlen + qlen);
    long long hits_total = 0, tiles_total = 0;
    Hsp *hd = nullptr;
    unsigned long long hcap = std::max<unsigned long long>(1ull << 16, (unsigned long long)cap);
    if (c->cap[SL_HSPS] / sizeof(Hsp) > hcap) hcap = c->cap[SL_HSPS] / sizeof(Hsp);
    for (int attempt = 0; attempt < 2; attempt++) {
        hits_total = tiles_total = 0;
        TRY(ensure_t(c, SL_HSPS, (size_t)hcap, &hd));
        CK(cudaMemsetAsync(&c->small->ctr, 0, sizeof(DevCounters), c->st));
        for (int s = 0; s < 2; s++) {
            if (!(params->strands & (1 << s))) continue;
            const uint32_t *Qs = s ? Qm : Qp;
            unsigned long long *starts = nullptr, total = 0;
            long long nq = 0;
            {
                Span sp(c, SFE_STAGE_COUNT);
                TRY(count_hits(c, v, Qs, qlen, &starts, &nq, &total));
            }
            hits_total += (long long)total;
            if (total == 0) continue;
            // query tiles of at most ~tile_hits hits each
            long long ntiles = (long long)((total + tile_hits - 1) / tile_hits);
            std::vector<long long> qb(ntiles + 1);
            std::vector<unsigned long long> hb(ntiles + 1);
            if (ntiles == 1) {
                qb[0] = 0;
                qb[1] = nq;
                hb[0] = 0;
                hb[1] = total;
            } else {
                long long *bd = nullptr;
                TRY(ensure_t(c, SL_BOUNDS, (size_t)(2 * (ntiles + 1)), &bd));
                unsigned long long *bs = reinterpret_cast<unsigned long long *>(bd + ntiles + 1);
                g_launches++;
                tile_bounds_kernel<<<(unsigned)((ntiles + 1 + 255) / 256), 256, 0, c->st>>>(
                    starts, nq, (unsigned long long)tile_hits, ntiles, bd, bs);
                CK(cudaGetLastError());
                CK(cudaMemcpyAsync(qb.data(), bd, (ntiles + 1) * 8, cudaMemcpyDeviceToHost, c->st));
                CK(cudaMemcpyAsync(hb.data(), bs, (ntiles + 1) * 8, cudaMemcpyDeviceToHost, c->st));
                CK(cudaStreamSynchronize(c->st));
            }
            unsigned long long maxtile = 0;
            for (long long k = 0; k < ntiles; k++) maxtile = std::max(maxtile, hb[k + 1] - hb[k]);
            if (maxtile >= (1ull << 32)) return fail(SFE_EINVAL, "a query tile exceeds 2^32 hits");
            int32_t *Ecarry = nullptr;
            if (ntiles > 1) {
                const long long nd = tlen + qlen;
                TRY(ensure_t(c, SL_ECARRY, (size_t)nd, &Ecarry));
                CK(cudaMemsetAsync(Ecarry, 0x80, (size_t)nd * 4, c->st));  // every E < 0
            }
            uint64_t *ha = nullptr, *hbuf = nullptr;
            void *tmp = nullptr;
            TRY(ensure_t(c, SL_HITS_A, (size_t)maxtile, &ha));
            TRY(ensure_t(c, SL_HITS_B, (size_t)maxtile, &hbuf));
            TRY(ensure(c, SL_TMP, radix_sort_temp_bytes((long long)maxtile), &tmp));
            const HitParams hp = hit_params(v, qlen);
            for (long long k = 0; k < ntiles; k++) {
                const long long nh = (long long)(hb[k + 1] - hb[k]);
                if (nh == 0) continue;
                tiles_total++;
                {
                    Span sp(c, SFE_STAGE_WRITE);
                    CK(launch_hit_write(Qs, hp, offs, pos, v.off2, v.pos2, qb[k], qb[k + 1],
                                        starts + qb[k], hb[k], (unsigned long long)nh, ha, c->st));
                }
                bool in_b = false;
                {
                    Span sp(c, SFE_STAGE_SORT);
                    CK(radix_sort(ha, hbuf, nullptr, nullptr, nh, 32, 32 + DB, tmp, &in_b, &c->small->status, c->st));
                }
                WalkSetup ws{Tp, tlen, Qs, qlen, s, pat.span, params, Ecarry, hd, hcap};
                ws.planes[0] = planes[s][0];
                ws.planes[1] = planes[s][1];
                TRY(walk_sorted(c, in_b ? hbuf : ha, nh, ws));
            }
        }
        TRY(sync_small(c));
        if (c->host_small->ctr.hsps <= hcap) break;
        hcap = c->host_small->ctr.hsps;  // grow and run again
    }
    Small sm = *c->host_small;
    TRY(check_status(sm.status | sm.ctr.status));
    fill_stats(sm, stats, hits_total, tiles_total);
    int r;
    {
        Span sp(c, SFE_STAGE_OUTPUT);
        r = finish_hsps(c, hd, sm.ctr.hsps, tlen, qlen, hsps, cap, nhsps);
    }
    CK(cudaStreamSynchronize(c->st));
    add_timings(c, stats);
    return r;
}

}  // extern "C"

// A batch of pairs: the pair table, the work items and the index buckets,
// fixed by the pairs' lengths and the seed.
struct BatchGeom {
    int npairs = 0;
    SeedPattern pat{};
    long long ttot = 0, qtot = 0, maxlen = 1, nbuckets = 0, titems = 0, qitems = 0;
    int dbits = 0, pbits = 0;
    std::vector<PairInfo> P;
    std::vector<long long> pref;  // target item prefix (npairs + 1), then query's
};

// Device buffers of one batch pipeline, and where its results end up.
struct BatchBufs {
    const uint8_t *tin = nullptr, *qin = nullptr;  // input bytes on the device
    unsigned char *meta = nullptr;                   // pair table + item prefixes
    uint32_t *tp = nullptr, *qp = nullptr, *qm = nullptr;  // packed (padded allocations)
    uint32_t *bcnt = nullptr, *boffs = nullptr;
    uint64_t *entries = nullptr;
    uint2 *slots = nullptr;  // index build scratch, one per target base
    uint64_t *ha = nullptr, *hb = nullptr;
    unsigned long long hitcap = 0;
    BatchHsp *hsps = nullptr;
    unsigned long long hcap = 0;
    uint4 *queue = nullptr;
    unsigned long long qcap = 0;
    void *tmp = nullptr;        // scans, sorts
    void *sched_tmp = nullptr;  // chunk schedule
    Small *small = nullptr;     // counters (scores set once)
    unsigned long long *nhits = nullptr;  // hit count the later stages use (0 on overflow)
    BatchHsp *sorted = nullptr;           // set by the pipeline
};

namespace {

int batch_geometry(const int64_t *toff, const int64_t *qoff, int npairs, const sfe_params *params,
                   BatchGeom &g) {
    if (!toff || !qoff) return fail(SFE_EINVAL, "toff or qoff is NULL");
    if (npairs < 1 || npairs > (1 << 16)) return fail(SFE_EINVAL, "npairs must be 1..65536");
    TRY(check_params(params));
    TRY(parse_pattern(params->seed_pattern, &g.pat));
    g.pat.step = params->step > 1 ? params->step : 1;
    if (toff[0] != 0 || qoff[0] != 0) return fail(SFE_EINVAL, "offsets must start at 0");
    long long maxsum = 1;
    g.maxlen = 1;
    for (int p = 0; p < npairs; p++) {
        const long long tl = toff[p + 1] - toff[p], ql = qoff[p + 1] - qoff[p];
        if (tl < 0 || ql < 0) return fail(SFE_EINVAL, "offsets must not decrease");
        if (tl >= (1LL << 20) || ql >= (1LL << 20))
            return fail(SFE_EINVAL, "batch sequences must be shorter than 2^20 bases");
        maxsum = std::max(maxsum, tl + ql);
        g.maxlen = std::max(g.maxlen, std::max(tl, ql));
    }
    g.npairs = npairs;
    g.ttot = toff[npairs];
    g.qtot = qoff[npairs];
    TRY(check_len(g.ttot, "concatenated target"));
    TRY(check_len(g.qtot, "concatenated query"));
    g.dbits = bits_for(maxsum);
    g.pbits = bits_for(npairs - 1);
    if (g.pbits + 1 + g.dbits > 32) return fail(SFE_EINVAL, "too many pairs for their lengths");
    g.P.assign(npairs, PairInfo{});
    g.nbuckets = 0;
    const int kbits = batch_table_bits(g.pat.weight);
    for (int p = 0; p < npairs; p++) {
        PairInfo &x = g.P[p];
        x.toff = toff[p];
        x.qoff = qoff[p];
        x.qoff_rc = g.qtot - qoff[p + 1];
        x.tlen = (int)(toff[p + 1] - toff[p]);
        x.qlen = (int)(qoff[p + 1] - qoff[p]);
        const long long npos = std::max(1LL, indexed_positions(g.pat, x.tlen));
        x.bbits = std::min(kbits, std::max(4, bits_for(npos - 1) - kBatchBucketShift));
        x.boff = g.nbuckets;
        x.pad = 0;
        g.nbuckets += 1LL << x.bbits;
    }
    // work items: chunks of one pair's target / query positions, pair by pair
    const int item = batch_item_size();
    g.pref.assign(2 * (size_t)(npairs + 1), 0);
    long long *tpref = g.pref.data(), *qpref = g.pref.data() + npairs + 1;
    for (int p = 0; p < npairs; p++) {
        const long long nt = std::max(0LL, (long long)g.P[p].tlen - g.pat.span + 1);
        const long long nq = std::max(0LL, (long long)g.P[p].qlen - g.pat.span + 1);
        tpref[p + 1] = tpref[p] + (nt + item - 1) / item;
        qpref[p + 1] = qpref[p] + 2 * ((nq + item - 1) / item);
    }
    g.titems = tpref[npairs];
    g.qitems = qpref[npairs];
    if (g.titems >= (1LL << 31) || g.qitems >= (1LL << 31))
        return fail(SFE_EINVAL, "batch too large");
    return SFE_OK;
}

size_t batch_meta_bytes(const BatchGeom &g) {
    return (((size_t)g.npairs * sizeof(PairInfo) + 255) & ~(size_t)255) + g.pref.size() * 8;
}

// Scratch shared by the scans and the sorts of a batch.
size_t batch_tmp_bytes(const BatchGeom &g, unsigned long long hitcap, unsigned long long hcap) {
    size_t t = std::max(scan_temp_bytes(2 * g.nbuckets), scan_temp_bytes(2 * g.qtot));
    t = std::max(t, radix_sort_temp_bytes((long long)hitcap));
    return std::max(t, batch_hsp_sort_temp_bytes((long long)hcap));
}

__global__ void guard_count_kernel(const unsigned long long *total, unsigned long long cap,
                                   unsigned long long *n) {
    *n = *total <= cap ? *total : 0ull;  // an overflowed hit list is not walked
}

// The whole batch on the device, without host synchronisation: pack, index,
// one-pass hit emission, sort, walk, HSP sort. Counts stay on the device
// (the sort, the walk and the HSP sort read them there), so the same calls
// run eagerly or are captured once into a CUDA graph. The pair table and the
// item prefixes must already be in b.meta and the scores in b.small.
int batch_pipeline(sfe_ctx *c, const BatchGeom &g, const sfe_params *params, BatchBufs &b) {
    cudaStream_t st = c->st;
    Small *sm = b.small;
    CK(cudaMemsetAsync(&sm->ctr, 0, sizeof(DevCounters), st));
    CK(cudaMemsetAsync(&sm->status, 0, 4, st));
    const size_t pbytes = ((size_t)g.npairs * sizeof(PairInfo) + 255) & ~(size_t)255;
    const PairInfo *dpairs = reinterpret_cast<const PairInfo *>(b.meta);
    const long long *dtpref = reinterpret_cast<const long long *>(b.meta + pbytes);
    const long long *dqpref = dtpref + g.npairs + 1;
    uint32_t *Tp = b.tp + SEQ_PAD, *Qp = b.qp + SEQ_PAD, *Qm = b.qm + SEQ_PAD;
    {
        Span sp(c, SFE_STAGE_PACK);
        CK(launch_pack(b.tin, g.ttot, params->input_codes, Tp, &sm->status, st));
        CK(launch_pack(b.qin, g.qtot, params->input_codes, Qp, &sm->status, st));
        CK(launch_revcomp(Qp, g.qtot, Qm, st));
    }
    {
        Span sp(c, SFE_STAGE_INDEX);
        CK(launch_batch_index(Tp, dpairs, dtpref, g.titems, g.npairs, g.pat, b.bcnt, g.nbuckets,
                              b.boffs, b.entries, b.slots, b.tmp, st));
    }
    {
        Span sp(c, SFE_STAGE_WRITE);
        CK(launch_batch_hit_emit(Qp, Qm, dpairs, dqpref, g.qitems, g.npairs, params->strands, g.pat,
                                 params->transition, g.dbits, g.nbuckets, b.boffs, b.entries,
                                 &sm->split, b.hitcap, b.ha, st));
        g_launches++;
        guard_count_kernel<<<1, 1, 0, st>>>(&sm->split, b.hitcap, b.nhits);
        CK(cudaGetLastError());
    }
    const long long cap = (long long)b.hitcap;
    uint64_t *ha = b.ha, *hb = b.hb;
    bool in_b = false;
    {
        Span sp(c, SFE_STAGE_SORT);
        // local t, then (pair, strand, diagonal): two stable passes, least significant first
        CK(radix_sort_dev(ha, hb, nullptr, nullptr, cap, b.nhits, 0, bits_for(g.maxlen), b.tmp,
                          &in_b, &sm->status, st));
        if (in_b) std::swap(ha, hb);
        CK(radix_sort_dev(ha, hb, nullptr, nullptr, cap, b.nhits, 32,
                          32 + g.pbits + 1 + g.dbits, b.tmp, &in_b, &sm->status, st));
    }
    const uint64_t *sorted = in_b ? hb : ha;
    WalkParams wp{};
    wp.T = Tp;
    wp.Q = Qp;
    wp.Qrc = Qm;
    wp.pairs = dpairs;
    wp.dbits = g.dbits;
    wp.span = g.pat.span;
    wp.xdrop = params->xdrop;
    wp.thresh = params->hsp_thresh;
    wp.flags = params->flags;
    wp.lane_cap = params->lane_cap > 0 ? params->lane_cap : DEFAULT_LANE_CAP;
    wp.scores = sm->scores;
    wp.bhsps = b.hsps;
    wp.hsp_cap = b.hcap;
    wp.ctr = &sm->ctr;
    wp.nd = b.nhits;
    TRY(walk_tiers(c, sorted, cap, wp, b.queue, b.qcap, params, sm, b.sched_tmp));
    {
        Span sp(c, SFE_STAGE_OUTPUT);
        CK(batch_hsp_sort(b.hsps, (long long)b.hcap, &sm->ctr.hsps, g.pbits, bits_for(g.maxlen),
                          b.tmp, &b.sorted, &sm->status, st));
    }
    return SFE_OK;
}

// Upper bound on hits in the first pass: the previous batch's count, or the
// chance count of the pairs' lengths (about 1.1e-6 per position pair and
// strand at 41% GC) with room for planted homology.
unsigned long long batch_hit_guess(const BatchGeom &g, unsigned long long hint) {
    double chance = 0.0;
    for (const PairInfo &x : g.P) chance += 2.2e-6 * (double)x.tlen * (double)x.qlen;
    const unsigned long long est = (unsigned long long)(3.0 * chance) + (1ull << 20);
    return std::max(hint, est);
}

// Report of a finished batch: status, stats, HSP count; copies the HSPs out.
int batch_finish(sfe_ctx *c, const BatchGeom &g, const BatchBufs &b, const Small &sm,
                 unsigned long long nhits, sfe_batch_hsp *hsps, int64_t cap, int64_t *nhsps,
                 sfe_stats *stats) {
    TRY(check_status(sm.status | sm.ctr.status));
    fill_stats(sm, stats, (long long)nhits, 1);
    const unsigned long long found = sm.ctr.hsps;
    *nhsps = (int64_t)found;
    if ((long long)found > cap) return fail(SFE_EOVERFLOW, "HSP buffer too small");
    if (found > 0) {
        const bool dev_out = is_device_ptr(hsps);
        CK(cudaMemcpyAsync(hsps, b.sorted, found * sizeof(BatchHsp),
                           dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
    }
    (void)g;
    return SFE_OK;
}

}  // namespace

extern "C" {

int sfe_run_batch(sfe_ctx *c, const uint8_t *targets, const int64_t *toff, const uint8_t *queries,
                  const int64_t *qoff, int32_t npairs, const sfe_params *params,
                  sfe_batch_hsp *hsps, int64_t cap, int64_t *nhsps, sfe_stats *stats) {
    if (!nhsps) return fail(SFE_EINVAL, "nhsps is NULL");
    BatchGeom g;
    TRY(batch_geometry(toff, qoff, npairs, params, g));
    TRY(begin(c, params->flags));
    TRY(upload_scores(c, params->scores));
    BatchBufs b;
    b.small = c->small;
    TRY(ensure_t(c, SL_PAIRS, batch_meta_bytes(g), &b.meta));
    const size_t pbytes = ((size_t)g.npairs * sizeof(PairInfo) + 255) & ~(size_t)255;
    CK(cudaMemcpyAsync(b.meta, g.P.data(), (size_t)npairs * sizeof(PairInfo),
                       cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(b.meta + pbytes, g.pref.data(), g.pref.size() * 8, cudaMemcpyHostToDevice,
                       c->st));
    {
        Span sp(c, SFE_STAGE_PACK);
        const void *tdev = nullptr, *qdev = nullptr;
        TRY(stage(c, SL_TIN, targets, (size_t)g.ttot, &tdev));
        TRY(stage(c, SL_QIN, queries, (size_t)g.qtot, &qdev));
        b.tin = reinterpret_cast<const uint8_t *>(tdev);
        b.qin = reinterpret_cast<const uint8_t *>(qdev);
    }
    TRY(ensure_t(c, SL_TP, packed_words(g.ttot), &b.tp));
    TRY(ensure_t(c, SL_QP, packed_words(g.qtot), &b.qp));
    TRY(ensure_t(c, SL_QM, packed_words(g.qtot), &b.qm));
    TRY(ensure_t(c, SL_BCOUNT, 2 * (size_t)g.nbuckets, &b.bcnt));
    TRY(ensure_t(c, SL_OFFS, 2 * (size_t)g.nbuckets + 1, &b.boffs));
    TRY(ensure_t(c, SL_BENTRIES, 2 * (size_t)std::max(1LL, g.ttot), &b.entries));
    TRY(ensure_t(c, SL_BSLOTS, (size_t)std::max(1LL, g.ttot), &b.slots));
    TRY(ensure_t(c, SL_BOUNDS, 1, &b.nhits));
    unsigned long long hitcap = batch_hit_guess(g, c->batch_hits_hint);
    unsigned long long hcap = std::max<unsigned long long>(1ull << 16, (unsigned long long)cap);
    if (c->cap[SL_HSPS] / sizeof(BatchHsp) > hcap) hcap = c->cap[SL_HSPS] / sizeof(BatchHsp);
    unsigned long long total = 0;
    for (int attempt = 0; attempt < 3; attempt++) {
        b.hitcap = hitcap;
        b.hcap = hcap;
        b.qcap = std::min<unsigned long long>(hitcap, kQueueMax);
        TRY(ensure_t(c, SL_HITS_A, (size_t)hitcap, &b.ha));
        TRY(ensure_t(c, SL_HITS_B, (size_t)hitcap, &b.hb));
        TRY(ensure_t(c, SL_HSPS, (size_t)hcap, &b.hsps));
        TRY(ensure_t(c, SL_QUEUE, (size_t)b.qcap, &b.queue));
        TRY(ensure(c, SL_TMP, batch_tmp_bytes(g, hitcap, hcap), &b.tmp));
        const uint32_t chunk = params->walk_chunk > 0 ? (uint32_t)params->walk_chunk
                                                      : walk_auto_chunk((long long)hitcap);
        if (params->walk_schedule != SFE_SCHED_NATURAL)
            TRY(ensure(c, SL_SCHED, walk_schedule_temp_bytes((long long)hitcap, chunk),
                       &b.sched_tmp));
        TRY(batch_pipeline(c, g, params, b));
        TRY(sync_small(c));
        total = c->host_small->split;
        const unsigned long long found = c->host_small->ctr.hsps;
        if (total <= hitcap && found <= hcap) break;
        if (total > hitcap) hitcap = total + total / 8;
        if (found > hcap) hcap = found;
        if (attempt == 2) return fail(SFE_ECUDA, "batch buffers kept overflowing");
    }
    c->batch_hits_hint = total + total / 16;
    if (total >= (1ull << 32)) return fail(SFE_EINVAL, "a batch may hold at most 2^32 - 1 hits");
    const Small sm = *c->host_small;
    const int r = batch_finish(c, g, b, sm, total, hsps, cap, nhsps, stats);
    CK(cudaStreamSynchronize(c->st));
    add_timings(c, stats);
    return r;
}

}  // extern "C"

// A batch captured once as a CUDA graph and replayed on new sequences of the
// same lengths. Every buffer the graph touches belongs to the plan.
struct sfe_batch_plan {
    sfe_ctx *c = nullptr;
    BatchGeom g;
    sfe_params p{};
    std::string pattern;
    BatchBufs b;
    uint8_t *tin = nullptr, *qin = nullptr;
    std::vector<void *> fixed;  // allocations that do not depend on the capacities
    std::vector<void *> sized;  // hits, HSPs, queue, scratch
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long launches = 0;  // kernels per replay
    Small *host_small = nullptr;      // pinned
};

namespace {

int plan_alloc(std::vector<void *> &list, size_t bytes, void **out) {
    void *q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(bytes, 256)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SFE_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    list.push_back(q);
    *out = q;
    return SFE_OK;
}

template <typename T>
int plan_alloc_t(std::vector<void *> &list, size_t count, T **out) {
    void *q = nullptr;
    TRY(plan_alloc(list, count * sizeof(T), &q));
    *out = reinterpret_cast<T *>(q);
    return SFE_OK;
}

void plan_drop_graph(sfe_batch_plan *pl) {
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    pl->exec = nullptr;
    pl->graph = nullptr;
}

void plan_drop_sized(sfe_batch_plan *pl) {
    for (void *q : pl->sized) cudaFree(q);
    pl->sized.clear();
}

// (Re)allocate the capacity-sized buffers and capture the pipeline.
int plan_capture(sfe_batch_plan *pl, unsigned long long hitcap, unsigned long long hcap) {
    sfe_ctx *c = pl->c;
    CK(cudaStreamSynchronize(c->st));
    plan_drop_graph(pl);
    plan_drop_sized(pl);
    BatchBufs &b = pl->b;
    b.hitcap = hitcap;
    b.hcap = hcap;
    b.qcap = std::min<unsigned long long>(hitcap, kQueueMax);
    TRY(plan_alloc_t(pl->sized, (size_t)hitcap, &b.ha));
    TRY(plan_alloc_t(pl->sized, (size_t)hitcap, &b.hb));
    TRY(plan_alloc_t(pl->sized, (size_t)hcap, &b.hsps));
    TRY(plan_alloc_t(pl->sized, (size_t)b.qcap, &b.queue));
    TRY(plan_alloc(pl->sized, batch_tmp_bytes(pl->g, hitcap, hcap), &b.tmp));
    b.sched_tmp = nullptr;
    if (pl->p.walk_schedule != SFE_SCHED_NATURAL) {
        const uint32_t chunk = pl->p.walk_chunk > 0 ? (uint32_t)pl->p.walk_chunk
                                                    : walk_auto_chunk((long long)hitcap);
        TRY(plan_alloc(pl->sized, walk_schedule_temp_bytes((long long)hitcap, chunk),
                       &b.sched_tmp));
    }
    c->tm.on = false;  // no event spans inside a graph
    const unsigned long long l0 = g_launches;
    CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeRelaxed));
    const int r = batch_pipeline(c, pl->g, &pl->p, b);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->st, &graph);
    pl->launches = g_launches - l0;
    g_launches = l0;  // captured, not launched
    if (r != SFE_OK) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return r;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SFE_ECUDA, std::string("graph capture failed: ") + cudaGetErrorString(e));
    }
    pl->graph = graph;
    CK(cudaGraphInstantiate(&pl->exec, graph, 0));
    return SFE_OK;
}

void plan_release(sfe_batch_plan *pl) {
    if (!pl) return;
    if (pl->c) {
        cudaSetDevice(pl->c->device);
        cudaStreamSynchronize(pl->c->st);
    }
    plan_drop_graph(pl);
    plan_drop_sized(pl);
    for (void *q : pl->fixed) cudaFree(q);
    if (pl->host_small) cudaFreeHost(pl->host_small);
    delete pl;
}

}  // namespace

// ------------------------------------------------------------- gapped stage

namespace {

// Boxes of the committed alignments, found through a grid of 1024 x 1024
// bases per strand: a box is listed in every grid cell it overlaps, and an
// anchor (t, q) is tested against the boxes of its own cell only. A box
// spanning more than kBigCells cells goes to a short list tested for every
// anchor instead. (A map by target start, scanning every box that starts
// within the longest box's length before t, spent about a second of host time
// on the 10 Mb pair's 231,379 anchors.)
struct CommittedBoxes {
    static constexpr int kG = 10;               // grid cell: 2^kG bases on each side
    static constexpr long long kBigCells = 4096;
    std::vector<sfe_galign> boxes;
    std::unordered_map<uint64_t, std::vector<int>> grid;
    std::vector<int> big;

    static uint64_t cell(int strand, int32_t t, int32_t q) {
        return ((uint64_t)(strand & 1) << 63) | ((uint64_t)(uint32_t)(t >> kG) << 32) |
               (uint64_t)(uint32_t)(q >> kG);
    }
    bool inside(const sfe_galign &b, int strand, int32_t t, int32_t q) const {
        return b.strand == strand && b.tstart <= t && t < b.tend && b.qstart <= q && q < b.qend;
    }
    bool contains(int strand, int32_t t, int32_t q) const {
        for (int id : big)
            if (inside(boxes[id], strand, t, q)) return true;
        const auto it = grid.find(cell(strand, t, q));
        if (it == grid.end()) return false;
        for (int id : it->second)
            if (inside(boxes[id], strand, t, q)) return true;
        return false;
    }
    void add(const sfe_galign &g) {
        const int id = (int)boxes.size();
        boxes.push_back(g);
        if (g.tend <= g.tstart || g.qend <= g.qstart) return;  // contains no anchor
        const int32_t t0 = g.tstart >> kG, t1 = (g.tend - 1) >> kG;
        const int32_t q0 = g.qstart >> kG, q1 = (g.qend - 1) >> kG;
        if ((long long)(t1 - t0 + 1) * (q1 - q0 + 1) > kBigCells) {
            big.push_back(id);
            return;
        }
        for (int32_t x = t0; x <= t1; x++)
            for (int32_t y = q0; y <= q1; y++)
                grid[cell(g.strand, x << kG, y << kG)].push_back(id);
    }
};

int check_ydrop_params(const sfe_ydrop_params *p) {
    if (!p) return fail(SFE_EINVAL, "params is NULL");
    for (int i = 0; i < 16; i++)
        if (p->scores[i] < -(1 << 15) || p->scores[i] > (1 << 15))
            return fail(SFE_EINVAL, "gapped scores must lie in [-2^15, 2^15]");
    if (p->gap_open < 0 || p->gap_extend < 0 || p->ydrop < 0 || p->gap_open > (1 << 28) ||
        p->gap_extend > (1 << 28) || p->ydrop > (1 << 28))
        return fail(SFE_EINVAL, "gap costs and ydrop must lie in [0, 2^28]");
    if (p->band < 0 || p->band > YD_MAX_BAND) return fail(SFE_EINVAL, "band must be 0..256");
    if (p->batch < 0) return fail(SFE_EINVAL, "batch must be >= 0");
    if (p->input_codes != 0 && p->input_codes != 1) return fail(SFE_EINVAL, "input_codes must be 0 or 1");
    return SFE_OK;
}

}  // namespace

extern "C" {

int sfe_ydrop_params_default(sfe_ydrop_params *p) {
    if (!p) return fail(SFE_EINVAL, "params is NULL");
    memset(p, 0, sizeof(*p));
    memcpy(p->scores, kHoxd70, sizeof(kHoxd70));
    p->gap_open = 400;
    p->gap_extend = 30;
    p->ydrop = 9400;
    p->gapped_thresh = 3000;
    p->band = YD_MAX_BAND;
    return SFE_OK;
}

int sfe_gapped_extend(sfe_ctx *c, const uint8_t *target, int64_t tlen, const uint8_t *query,
                      int64_t qlen, const sfe_hsp *hsps, int64_t nhsps,
                      const sfe_ydrop_params *params, sfe_galign *out, int64_t cap,
                      int64_t *nout, sfe_ydrop_stats *stats) {
    const auto w0 = std::chrono::steady_clock::now();
    if (!nout) return fail(SFE_EINVAL, "nout is NULL");
    TRY(check_ydrop_params(params));
    TRY(check_len(tlen, "target"));
    TRY(check_len(qlen, "query"));
    if (nhsps < 0 || nhsps >= (1LL << 31)) return fail(SFE_EINVAL, "nhsps out of range");
    if (nhsps > 0 && !hsps) return fail(SFE_EINVAL, "hsps is NULL");
    TRY(begin(c));
    // the anchors, on the host: the scan and the commit run there
    std::vector<sfe_hsp> H((size_t)nhsps);
    if (nhsps > 0) {
        if (is_device_ptr(hsps)) {
            CK(cudaMemcpyAsync(H.data(), hsps, (size_t)nhsps * sizeof(sfe_hsp),
                               cudaMemcpyDeviceToHost, c->st));
            CK(cudaStreamSynchronize(c->st));
        } else {
            memcpy(H.data(), hsps, (size_t)nhsps * sizeof(sfe_hsp));
        }
    }
    for (const sfe_hsp &h : H)
        if ((h.strand != 0 && h.strand != 1) || h.len < 0 || h.tpos < 0 || h.qpos < 0 ||
            (int64_t)h.tpos + h.len / 2 > tlen || (int64_t)h.qpos + h.len / 2 > qlen)
            return fail(SFE_EINVAL, "an HSP's anchor lies outside the sequences");
    std::vector<int> order((size_t)nhsps);
    for (int k = 0; k < (int)nhsps; k++) order[k] = k;
    std::sort(order.begin(), order.end(), [&](int x, int y) {
        const sfe_hsp &a = H[x], &b = H[y];
        if (a.score != b.score) return a.score > b.score;
        if (a.strand != b.strand) return a.strand < b.strand;
        if (a.tpos != b.tpos) return a.tpos < b.tpos;
        if (a.qpos != b.qpos) return a.qpos < b.qpos;
        return a.len < b.len;
    });
    // the sequences, packed on the device
    uint32_t *Tp = nullptr, *Qp = nullptr, *Qm = nullptr;
    const void *tdev = nullptr, *qdev = nullptr;
    TRY(stage(c, SL_TIN, target, (size_t)tlen, &tdev));
    TRY(stage(c, SL_QIN, query, (size_t)qlen, &qdev));
    TRY(pack_slot(c, SL_TP, reinterpret_cast<const uint8_t *>(tdev), tlen, params->input_codes,
                  &Tp));
    TRY(pack_slot(c, SL_QP, reinterpret_cast<const uint8_t *>(qdev), qlen, params->input_codes,
                  &Qp));
    TRY(rc_slot(c, SL_QM, Qp, qlen, &Qm));
    TRY(sync_small(c));
    TRY(check_status(c->host_small->status));
    YdParams yp;
    memcpy(yp.scores, params->scores, sizeof(yp.scores));
    yp.gap_open = params->gap_open;
    yp.gap_extend = params->gap_extend;
    yp.ydrop = params->ydrop;
    yp.band = params->band > 0 ? params->band : YD_MAX_BAND;
    const long long K = params->batch > 0 ? std::min<long long>(params->batch, nhsps) : nhsps;
    int4 *dan = nullptr;
    YdHalf *dhalf = nullptr;
    TRY(ensure_t(c, SL_YANCH, (size_t)std::max(1LL, K), &dan));
    TRY(ensure_t(c, SL_YHALF, (size_t)std::max(1LL, 2 * K), &dhalf));
    std::vector<int4> ban;
    std::vector<int> bidx;
    std::vector<YdHalf> half, hlaunch;
    std::vector<int4> blaunch;
    std::vector<int> lorder;
    ban.reserve((size_t)K);
    bidx.reserve((size_t)K);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    CK(cudaEventCreate(&ev[0]));
    CK(cudaEventCreate(&ev[1]));
    CommittedBoxes com;
    sfe_ydrop_stats st{};
    st.anchors = nhsps;
    uint32_t status = 0;
    int rc = SFE_OK;
    size_t j = 0;
    while (j < order.size() && rc == SFE_OK) {
        // phase 1: the next anchors not contained in what is committed
        ban.clear();
        bidx.clear();
        while ((long long)ban.size() < K && j < order.size()) {
            const sfe_hsp &h = H[order[j]];
            const int32_t ta = h.tpos + h.len / 2, qa = h.qpos + h.len / 2;
            if (com.contains(h.strand, ta, qa))
                st.skipped++;
            else {
                ban.push_back(make_int4(h.strand, ta, qa, 0));
                bidx.push_back(order[j]);
            }
            j++;
        }
        if (ban.empty()) break;
        st.batches++;
        // phase 2: every anchor of the batch, both halves, on the GPU. The
        // warps start in launch order, so the anchors of the longest ungapped
        // HSPs (those in long homologous regions, whose extensions run far)
        // go first and a long extension does not start at the end of the
        // batch; the results come back in the batch's order for the commit.
        const int nb = (int)ban.size();
        half.resize(2 * (size_t)nb);
        lorder.resize((size_t)nb);
        for (int b = 0; b < nb; b++) lorder[b] = b;
        std::stable_sort(lorder.begin(), lorder.end(),
                         [&](int x, int y) { return H[bidx[x]].len > H[bidx[y]].len; });
        blaunch.resize((size_t)nb);
        for (int k = 0; k < nb; k++) blaunch[k] = ban[lorder[k]];
        hlaunch.resize(2 * (size_t)nb);
        cudaError_t e = cudaMemcpyAsync(dan, blaunch.data(), nb * sizeof(int4),
                                        cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], c->st);
        if (e == cudaSuccess) e = launch_ydrop(Tp, tlen, Qp, Qm, qlen, dan, nb, yp, dhalf, c->st);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hlaunch.data(), dhalf, 2 * (size_t)nb * sizeof(YdHalf),
                                cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e == cudaSuccess)
            for (int k = 0; k < nb; k++) {
                half[2 * (size_t)lorder[k]] = hlaunch[2 * (size_t)k];
                half[2 * (size_t)lorder[k] + 1] = hlaunch[2 * (size_t)k + 1];
            }
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = fail(SFE_ECUDA, std::string("gapped extension: ") + cudaGetErrorString(e));
            break;
        }
        st.device_ms += ms;
        // phase 3: commit in order
        for (int b = 0; b < nb; b++) {
            const YdHalf &f = half[2 * b], &r = half[2 * b + 1];
            status |= f.status | r.status;
            const int4 an = ban[b];
            const long long work = f.cells + r.cells;
            if (b > 0 && com.contains(an.x, an.y, an.z)) {
                st.shadow++;
                st.shadow_cells += work;
                continue;
            }
            st.extended++;
            st.cells += work;
            const long long score = (long long)f.best + r.best;
            if (score > INT_MAX) status |= ST_SCORE_OVERFLOW;
            if (score >= params->gapped_thresh) {
                sfe_galign g;
                g.strand = an.x;
                g.tstart = an.y - r.bi;
                g.tend = an.y + f.bi;
                g.qstart = an.z - r.bj;
                g.qend = an.z + f.bj;
                g.score = (int32_t)score;
                com.add(g);
            }
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc != SFE_OK) return rc;
    if (status & ST_SCORE_OVERFLOW) return fail(SFE_EOVERFLOW, "a gapped score left the int32 range");
    std::vector<sfe_galign> &A = com.boxes;
    std::sort(A.begin(), A.end(), [](const sfe_galign &x, const sfe_galign &y) {
        if (x.strand != y.strand) return x.strand < y.strand;
        if (x.tstart != y.tstart) return x.tstart < y.tstart;
        if (x.qstart != y.qstart) return x.qstart < y.qstart;
        if (x.tend != y.tend) return x.tend < y.tend;
        if (x.qend != y.qend) return x.qend < y.qend;
        return x.score < y.score;
    });
    st.committed = (int64_t)A.size();
    *nout = st.committed;
    st.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0)
                      .count();
    if (stats) *stats = st;
    if ((int64_t)A.size() > cap) return fail(SFE_EOVERFLOW, "alignment buffer too small");
    if (!A.empty()) {
        CK(cudaMemcpyAsync(out, A.data(), A.size() * sizeof(sfe_galign),
                           is_device_ptr(out) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost,
                           c->st));
        CK(cudaStreamSynchronize(c->st));
    }
    return SFE_OK;
}

int sfe_test_committed_boxes(const sfe_galign *boxes, int64_t n, const int32_t *queries,
                             int64_t m, uint8_t *inside) {
    if (n < 0 || m < 0) return fail(SFE_EINVAL, "negative count");
    if ((n > 0 && !boxes) || (m > 0 && (!queries || !inside)))
        return fail(SFE_EINVAL, "boxes, queries or inside is NULL");
    CommittedBoxes com;
    for (int64_t k = 0; k < n; k++) com.add(boxes[k]);
    for (int64_t k = 0; k < m; k++)
        inside[k] = com.contains(queries[3 * k], queries[3 * k + 1], queries[3 * k + 2]) ? 1 : 0;
    return SFE_OK;
}

}  // extern "C"

extern "C" {

int sfe_batch_plan_create(sfe_ctx *c, const int64_t *toff, const int64_t *qoff, int32_t npairs,
                          const sfe_params *params, int64_t hit_cap, sfe_batch_plan **out) {
    if (!out) return fail(SFE_EINVAL, "out is NULL");
    *out = nullptr;
    if (hit_cap < 0) return fail(SFE_EINVAL, "hit_cap must be >= 0");
    BatchGeom g;
    TRY(batch_geometry(toff, qoff, npairs, params, g));
    if (params->flags & SFE_TIME_STAGES)
        return fail(SFE_EINVAL, "SFE_TIME_STAGES is not available in a captured batch");
    TRY(begin(c));
    sfe_batch_plan *pl = new sfe_batch_plan;
    pl->c = c;
    pl->g = std::move(g);
    pl->p = *params;
    pl->pattern = params->seed_pattern ? params->seed_pattern : kDefaultPattern;
    pl->p.seed_pattern = pl->pattern.c_str();
    auto bail = [&](int r) {
        plan_release(pl);
        return r;
    };
    BatchBufs &b = pl->b;
    const BatchGeom &G = pl->g;
    int r = SFE_OK;
    if (cudaMallocHost(&pl->host_small, sizeof(Small)) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(SFE_ENOMEM, "pinned allocation failed"));
    }
    if ((r = plan_alloc_t(pl->fixed, 1, &b.small)) != SFE_OK) return bail(r);
    if ((r = plan_alloc_t(pl->fixed, 1, &b.nhits)) != SFE_OK) return bail(r);
    if ((r = plan_alloc_t(pl->fixed, batch_meta_bytes(G), &b.meta)) != SFE_OK) return bail(r);
    if ((r = plan_alloc_t(pl->fixed, (size_t)std::max(1LL, G.ttot), &pl->tin)) != SFE_OK ||
        (r = plan_alloc_t(pl->fixed, (size_t)std::max(1LL, G.qtot), &pl->qin)) != SFE_OK ||
        (r = plan_alloc_t(pl->fixed, packed_words(G.ttot), &b.tp)) != SFE_OK ||
        (r = plan_alloc_t(pl->fixed, packed_words(G.qtot), &b.qp)) != SFE_OK ||
        (r = plan_alloc_t(pl->fixed, packed_words(G.qtot), &b.qm)) != SFE_OK ||
        (r = plan_alloc_t(pl->fixed, 2 * (size_t)G.nbuckets, &b.bcnt)) != SFE_OK ||
        (r = plan_alloc_t(pl->fixed, 2 * (size_t)G.nbuckets + 1, &b.boffs)) != SFE_OK ||
        (r = plan_alloc_t(pl->fixed, 2 * (size_t)std::max(1LL, G.ttot), &b.entries)) != SFE_OK ||
        (r = plan_alloc_t(pl->fixed, (size_t)std::max(1LL, G.ttot), &b.slots)) != SFE_OK)
        return bail(r);
    b.tin = pl->tin;
    b.qin = pl->qin;
    const size_t pbytes = ((size_t)G.npairs * sizeof(PairInfo) + 255) & ~(size_t)255;
    if (cudaMemsetAsync(b.small, 0, sizeof(Small), c->st) != cudaSuccess ||
        cudaMemcpyAsync(b.small->scores, params->scores, 64, cudaMemcpyHostToDevice, c->st) !=
            cudaSuccess ||
        cudaMemcpyAsync(b.meta, G.P.data(), (size_t)G.npairs * sizeof(PairInfo),
                        cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaMemcpyAsync(b.meta + pbytes, G.pref.data(), G.pref.size() * 8, cudaMemcpyHostToDevice,
                        c->st) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(SFE_ECUDA, "plan set-up copies failed"));
    }
    const unsigned long long hitcap =
        hit_cap > 0 ? (unsigned long long)hit_cap : batch_hit_guess(G, c->batch_hits_hint);
    if ((r = plan_capture(pl, hitcap, 1ull << 16)) != SFE_OK) return bail(r);
    *out = pl;
    return SFE_OK;
}

void sfe_batch_plan_free(sfe_batch_plan *pl) { plan_release(pl); }

int sfe_batch_plan_run(sfe_batch_plan *pl, const uint8_t *targets, const uint8_t *queries,
                       sfe_batch_hsp *hsps, int64_t cap, int64_t *nhsps, sfe_stats *stats) {
    if (!pl || !nhsps) return fail(SFE_EINVAL, "plan or nhsps is NULL");
    sfe_ctx *c = pl->c;
    TRY(begin(c));
    const BatchGeom &G = pl->g;
    if ((G.ttot > 0 && !targets) || (G.qtot > 0 && !queries))
        return fail(SFE_EINVAL, "input pointer is NULL");
    if (G.ttot > 0)
        CK(cudaMemcpyAsync(pl->tin, targets, (size_t)G.ttot,
                           is_device_ptr(targets) ? cudaMemcpyDeviceToDevice
                                                  : cudaMemcpyHostToDevice,
                           c->st));
    if (G.qtot > 0)
        CK(cudaMemcpyAsync(pl->qin, queries, (size_t)G.qtot,
                           is_device_ptr(queries) ? cudaMemcpyDeviceToDevice
                                                  : cudaMemcpyHostToDevice,
                           c->st));
    unsigned long long total = 0, launches = 0;
    for (int attempt = 0; attempt < 3; attempt++) {
        CK(cudaGraphLaunch(pl->exec, c->st));
        launches += pl->launches;
        CK(cudaMemcpyAsync(pl->host_small, pl->b.small, sizeof(Small), cudaMemcpyDeviceToHost,
                           c->st));
        CK(cudaStreamSynchronize(c->st));
        total = pl->host_small->split;
        const unsigned long long found = pl->host_small->ctr.hsps;
        if (total <= pl->b.hitcap && found <= pl->b.hcap) break;
        if (attempt == 2) return fail(SFE_ECUDA, "batch buffers kept overflowing");
        // grow and capture again (the inputs are still in the plan's buffers)
        TRY(plan_capture(pl, std::max(pl->b.hitcap, total + total / 8),
                         std::max(pl->b.hcap, found)));
    }
    c->batch_hits_hint = total + total / 16;
    const Small sm = *pl->host_small;
    const int r = batch_finish(c, G, pl->b, sm, total, hsps, cap, nhsps, stats);
    CK(cudaStreamSynchronize(c->st));
    if (stats) stats->launches = (int64_t)launches;
    g_launches += launches;
    return r;
}

// ---------------------------------------------------------------------------
// Work predictor: training data, loss/gradient, Adam, FP16 inference.

int32_t sfe_mlp_param_count(void) { return mlp_param_count(); }
int64_t sfe_mlp_model_bytes(void) { return (int64_t)mlp_model_bytes(); }

int sfe_mlp_init(sfe_ctx *c, float *params, uint64_t seed) {
    TRY(begin(c));
    if (!is_device_ptr(params)) return fail(SFE_EINVAL, "params must be device memory");
    CK(launch_mlp_init(params, (unsigned long long)seed, c->st));
    CK(cudaStreamSynchronize(c->st));
    return SFE_OK;
}

int sfe_mlp_pack(sfe_ctx *c, const float *params, void *model) {
    TRY(begin(c));
    if (!is_device_ptr(params) || !is_device_ptr(model))
        return fail(SFE_EINVAL, "params and model must be device memory");
    CK(launch_mlp_pack(params, model, c->st));
    CK(cudaStreamSynchronize(c->st));
    return SFE_OK;
}

}  // extern "C"

struct sfe_mlp_data {
    int device = 0;
    long long n = 0;
    int npairs = 0;
    int span = 19;  // seed span of the run that logged the records
    long long ttot = 0, qtot = 0;
    uint32_t *tp = nullptr, *qp = nullptr, *qm = nullptr;  // packed, with padding
    PairInfo *pairs = nullptr;
    sfe_ext_record *recs = nullptr;
    // training scratch
    uint64_t *ka = nullptr, *kb = nullptr;
    uint32_t *perm = nullptr;
    void *tmp = nullptr;
    float *grad = nullptr, *m = nullptr, *v = nullptr;
    double *loss = nullptr;  // one per epoch (grown on demand)
    int loss_cap = 0;
    uint32_t *status = nullptr;
    std::vector<void *> owned;
};

namespace {

int data_alloc(sfe_mlp_data *d, size_t bytes, void **out) {
    void *p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SFE_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    d->owned.push_back(p);
    *out = p;
    return SFE_OK;
}

template <typename T>
int data_alloc_t(sfe_mlp_data *d, size_t count, T **out) {
    void *p = nullptr;
    TRY(data_alloc(d, count * sizeof(T), &p));
    *out = reinterpret_cast<T *>(p);
    return SFE_OK;
}

void data_release(sfe_mlp_data *d) {
    if (!d) return;
    cudaSetDevice(d->device);
    for (void *p : d->owned) cudaFree(p);
    delete d;
}

// Pack (host or device) bases into a new padded buffer owned by d.
int data_pack(sfe_ctx *c, sfe_mlp_data *d, const uint8_t *src, long long n, int codes,
              uint32_t **base0) {
    uint32_t *a = nullptr;
    TRY(data_alloc_t(d, packed_words(n), &a));
    CK(cudaMemsetAsync(a, 0, packed_words(n) * 4, c->st));
    *base0 = a + SEQ_PAD;
    if (n == 0) return SFE_OK;
    const uint8_t *dev = src;
    if (!is_device_ptr(src)) {
        uint8_t *stg = nullptr;
        TRY(data_alloc_t(d, (size_t)n, &stg));
        CK(cudaMemcpyAsync(stg, src, (size_t)n, cudaMemcpyHostToDevice, c->st));
        dev = stg;
    }
    CK(launch_pack(dev, n, codes, *base0, d->status, c->st));
    return SFE_OK;
}

int data_status(sfe_ctx *c, sfe_mlp_data *d) {
    uint32_t st = 0;
    CK(cudaMemcpyAsync(&st, d->status, 4, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (st & ST_BAD_HIT) return fail(SFE_EINVAL, "a record's pair or strand is out of range");
    return check_status(st);
}

int data_check(sfe_ctx *c, const sfe_mlp_data *d) {
    if (!d) return fail(SFE_EINVAL, "data is NULL");
    if (d->device != c->device) return fail(SFE_EINVAL, "data belongs to another device");
    return SFE_OK;
}

}  // namespace

extern "C" {

int sfe_mlp_data_create(sfe_ctx *c, const uint8_t *targets, const int64_t *toff,
                        const uint8_t *queries, const int64_t *qoff, int32_t npairs,
                        int32_t input_codes, int32_t span, const sfe_ext_record *recs, int64_t n,
                        sfe_mlp_data **out) {
    if (!out || !toff || !qoff) return fail(SFE_EINVAL, "out, toff or qoff is NULL");
    *out = nullptr;
    if (npairs < 1 || npairs > (1 << 16)) return fail(SFE_EINVAL, "npairs must be 1..65536");
    if (n < 0 || n >= (1LL << 32)) return fail(SFE_EINVAL, "record count must be in [0, 2^32)");
    if (n > 0 && !recs) return fail(SFE_EINVAL, "recs is NULL");
    if (input_codes != 0 && input_codes != 1) return fail(SFE_EINVAL, "input_codes must be 0 or 1");
    if (span < 1 || span > MAX_SPAN) return fail(SFE_EINVAL, "span must be in [1, 32]");
    if (toff[0] != 0 || qoff[0] != 0) return fail(SFE_EINVAL, "offsets must start at 0");
    for (int p = 0; p < npairs; p++)
        if (toff[p + 1] < toff[p] || qoff[p + 1] < qoff[p])
            return fail(SFE_EINVAL, "offsets must not decrease");
    TRY(check_len(toff[npairs], "concatenated target"));
    TRY(check_len(qoff[npairs], "concatenated query"));
    TRY(begin(c));
    sfe_mlp_data *d = new sfe_mlp_data;
    d->device = c->device;
    d->n = n;
    d->npairs = npairs;
    d->span = span;
    d->ttot = toff[npairs];
    d->qtot = qoff[npairs];
    auto bail = [&](int r) {
        cudaStreamSynchronize(c->st);
        data_release(d);
        return r;
    };
    int r = SFE_OK;
    if ((r = data_alloc_t(d, 1, &d->status)) != SFE_OK) return bail(r);
    if (cudaMemsetAsync(d->status, 0, 4, c->st) != cudaSuccess) return bail(fail(SFE_ECUDA, "memset"));
    std::vector<PairInfo> P(npairs);
    for (int p = 0; p < npairs; p++) {
        P[p] = PairInfo{};
        P[p].toff = toff[p];
        P[p].qoff = qoff[p];
        P[p].qoff_rc = d->qtot - qoff[p + 1];
        P[p].tlen = (int)(toff[p + 1] - toff[p]);
        P[p].qlen = (int)(qoff[p + 1] - qoff[p]);
    }
    if ((r = data_alloc_t(d, (size_t)npairs, &d->pairs)) != SFE_OK) return bail(r);
    if (cudaMemcpyAsync(d->pairs, P.data(), (size_t)npairs * sizeof(PairInfo),
                        cudaMemcpyHostToDevice, c->st) != cudaSuccess)
        return bail(fail(SFE_ECUDA, "copy of the pair table failed"));
    if ((r = data_pack(c, d, targets, d->ttot, input_codes, &d->tp)) != SFE_OK) return bail(r);
    if ((r = data_pack(c, d, queries, d->qtot, input_codes, &d->qp)) != SFE_OK) return bail(r);
    uint32_t *qm_alloc = nullptr;
    if ((r = data_alloc_t(d, packed_words(d->qtot), &qm_alloc)) != SFE_OK) return bail(r);
    d->qm = qm_alloc + SEQ_PAD;
    if (launch_revcomp(d->qp, d->qtot, d->qm, c->st) != cudaSuccess)
        return bail(fail(SFE_ECUDA, "reverse complement failed"));
    if ((r = data_alloc_t(d, (size_t)std::max<int64_t>(n, 1), &d->recs)) != SFE_OK) return bail(r);
    if (n > 0 &&
        cudaMemcpyAsync(d->recs, recs, (size_t)n * sizeof(sfe_ext_record),
                        is_device_ptr(recs) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        c->st) != cudaSuccess)
        return bail(fail(SFE_ECUDA, "copy of the records failed"));
    if (launch_validate_records(d->recs, n, npairs, d->status, c->st) != cudaSuccess)
        return bail(fail(SFE_ECUDA, "record check failed"));
    if ((r = data_status(c, d)) != SFE_OK) return bail(r);
    *out = d;
    return SFE_OK;
}

void sfe_mlp_data_free(sfe_mlp_data *d) { data_release(d); }

int sfe_mlp_loss_grad(sfe_ctx *c, const sfe_mlp_data *d, const float *params, float *grad,
                      float *preds, double *loss) {
    TRY(begin(c));
    TRY(data_check(c, d));
    if (!loss) return fail(SFE_EINVAL, "loss is NULL");
    if (!is_device_ptr(params) || (grad && !is_device_ptr(grad)) ||
        (preds && !is_device_ptr(preds)))
        return fail(SFE_EINVAL, "params, grad and preds must be device memory");
    double *dl = nullptr;
    TRY(ensure_t(c, SL_TMP, 1, &dl));
    CK(cudaMemsetAsync(dl, 0, 8, c->st));
    if (grad) CK(cudaMemsetAsync(grad, 0, (size_t)mlp_param_count() * 4, c->st));
    CK(launch_mlp_fwd_bwd(d->tp, d->ttot, d->qp, d->qm, d->qtot, d->pairs, d->span, d->recs, nullptr,
                          d->n, params, grad, preds, dl, c->st));
    double h = 0.0;
    CK(cudaMemcpyAsync(&h, dl, 8, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    *loss = d->n > 0 ? h / (double)d->n : 0.0;
    return SFE_OK;
}

int sfe_mlp_predict(sfe_ctx *c, const sfe_mlp_data *d, const void *model, float *preds) {
    TRY(begin(c));
    TRY(data_check(c, d));
    if (!is_device_ptr(model) || (d->n > 0 && !is_device_ptr(preds)))
        return fail(SFE_EINVAL, "model and preds must be device memory");
    CK(launch_mlp_predict16(d->tp, d->ttot, d->qp, d->qm, d->qtot, d->pairs, d->span, d->recs,
                            d->n, model, preds, c->st));
    CK(cudaStreamSynchronize(c->st));
    return SFE_OK;
}

int sfe_mlp_train(sfe_ctx *c, const sfe_mlp_data *dc, float *params, int32_t epochs,
                  int32_t batch, float lr, uint64_t seed, double *epoch_loss) {
    TRY(begin(c));
    TRY(data_check(c, dc));
    sfe_mlp_data *d = const_cast<sfe_mlp_data *>(dc);  // training scratch lives in the handle
    if (!is_device_ptr(params)) return fail(SFE_EINVAL, "params must be device memory");
    if (epochs < 0 || batch < 1 || !(lr > 0.f)) return fail(SFE_EINVAL, "bad epochs, batch or lr");
    const long long n = d->n;
    if (n == 0 || epochs == 0) return SFE_OK;
    const int np = mlp_param_count();
    if (!d->grad) {
        TRY(data_alloc_t(d, (size_t)np, &d->grad));
        TRY(data_alloc_t(d, (size_t)np, &d->m));
        TRY(data_alloc_t(d, (size_t)np, &d->v));
        TRY(data_alloc_t(d, (size_t)n, &d->ka));
        TRY(data_alloc_t(d, (size_t)n, &d->kb));
        TRY(data_alloc_t(d, (size_t)n, &d->perm));
        TRY(data_alloc(d, radix_sort_temp_bytes(n), &d->tmp));
    }
    if (d->loss_cap < epochs) {
        TRY(data_alloc_t(d, (size_t)epochs, &d->loss));
        d->loss_cap = epochs;
    }
    CK(cudaMemsetAsync(d->m, 0, (size_t)np * 4, c->st));
    CK(cudaMemsetAsync(d->v, 0, (size_t)np * 4, c->st));
    CK(cudaMemsetAsync(d->loss, 0, (size_t)epochs * 8, c->st));
    CK(cudaMemsetAsync(d->status, 0, 4, c->st));
    int step = 0;
    for (int e = 0; e < epochs; e++) {
        CK(launch_perm(n, (unsigned long long)seed, e, d->ka, d->kb, d->tmp, d->perm, d->status,
                       c->st));
        for (long long b0 = 0; b0 < n; b0 += batch) {
            const long long nb = std::min<long long>(batch, n - b0);
            CK(cudaMemsetAsync(d->grad, 0, (size_t)np * 4, c->st));
            CK(launch_mlp_fwd_bwd(d->tp, d->ttot, d->qp, d->qm, d->qtot, d->pairs, d->span,
                                  d->recs, d->perm + b0, nb, params, d->grad, nullptr,
                                  d->loss + e, c->st));
            CK(launch_adam(params, d->grad, d->m, d->v, lr, ++step, c->st));
        }
    }
    std::vector<double> h((size_t)epochs);
    CK(cudaMemcpyAsync(h.data(), d->loss, (size_t)epochs * 8, cudaMemcpyDeviceToHost, c->st));
    TRY(data_status(c, d));
    if (epoch_loss)
        for (int e = 0; e < epochs; e++) epoch_loss[e] = h[(size_t)e] / (double)n;
    return SFE_OK;
}

}  // extern "C"
