// sfe_ungapped_xdrop_static: the hit-list skip + X-drop call for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's memory pool or under a strict memory budget, plugins loaded into
// a host that owns every device allocation, and real-time paths where an
// allocation (and the synchronisation it may imply) is not allowed. For them
// this call keeps all of its scratch in one file-scope device array, sized
// once at load time and held by every GPU that loads the library until the
// process exits. The caller still provides every input and output buffer.
#include <algorithm>
#include <climits>
#include <cstring>

#include "sfe_internal.cuh"

namespace {

using namespace sfe;

// Limits of the static scratch (the call rejects larger inputs with SFE_ELIMIT).
constexpr long long kMaxBases = 1LL << 20;  // per sequence
constexpr long long kMaxHits = 1LL << 17;
constexpr int kMaxDevices = 64;

// Layout of the scratch array (offsets in bytes, 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kPackedBytes = align256(((kMaxBases + 15) / 16 + 2 * SEQ_PAD) * 4);
struct StaticSmall {
    int32_t scores[16];
    DevCounters ctr;
    uint32_t status;
    uint32_t queue_len;
    unsigned long long split;
};
constexpr size_t kOffSmall = 0;
constexpr size_t kOffT = align256(sizeof(StaticSmall));
constexpr size_t kOffQ = kOffT + kPackedBytes;
constexpr size_t kOffQm = kOffQ + kPackedBytes;
constexpr size_t kOffKeysA = kOffQm + kPackedBytes;
constexpr size_t kOffKeysB = kOffKeysA + align256(kMaxHits * 8);
constexpr size_t kOffQueue = kOffKeysB + align256(kMaxHits * 8);
constexpr size_t kOffTmp = kOffQueue + align256(kMaxHits * 16);
constexpr size_t kTmpBytes = 8u << 20;  // radix-sort and HSP-sort temporaries
constexpr size_t kStaticBytes = kOffTmp + kTmpBytes;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Host-side device addresses of g_static_scratch, one per device. In host
// code the symbol itself is only a stand-in, not a device address. Atomic:
// two host threads making their first call on a device at the same time
// both look the address up and store the same value.
std::atomic<void *> g_scratch_addr[kMaxDevices];

int scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return SFE_EINVAL;
    void *p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) {
            cudaGetLastError();
            return SFE_ECUDA;
        }
        g_scratch_addr[dev].store(p, std::memory_order_release);
    }
    *out = reinterpret_cast<unsigned char *>(p);
    return SFE_OK;
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int parse(const char *s, SeedPattern *p) {
    if (!s) s = "1110100110010101111";
    const int n = (int)strlen(s);
    if (n < 1 || n > MAX_SPAN) return SFE_EINVAL;
    memset(p, 0, sizeof(*p));
    p->span = n;
    p->step = 1;
    for (int i = 0; i < n; i++) {
        if (s[i] == '1')
            p->care[p->weight++] = i;
        else if (s[i] != '0')
            return SFE_EINVAL;
    }
    return (p->weight >= 1 && p->weight <= MAX_WEIGHT) ? SFE_OK : SFE_EINVAL;
}

int bits_of(long long v) {
    int b = 1;
    while (b < 63 && (1LL << b) <= v) b++;
    return b;
}

__global__ void static_split_kernel(const uint64_t *keys, long long n, unsigned long long *split) {
    long long lo = 0, hi = n;  // first index with the strand bit set
    while (lo < hi) {
        const long long mid = (lo + hi) / 2;
        if ((keys[mid] >> 63) == 0)
            lo = mid + 1;
        else
            hi = mid;
    }
    *split = (unsigned long long)lo;
}

int device_status(uint32_t st) {
    if (st & (ST_BAD_SYMBOL | ST_BAD_HIT)) return SFE_EINVAL;
    if (st & ST_SCORE_OVERFLOW) return SFE_EOVERFLOW;
    if (st & ST_TIMEOUT) return SFE_ETIMEOUT;
    return SFE_OK;
}

#define SCK(x)                          \
    do {                                \
        if ((x) != cudaSuccess) {       \
            cudaGetLastError();         \
            return SFE_ECUDA;           \
        }                               \
    } while (0)

}  // namespace

extern "C" int sfe_ungapped_xdrop_static(const uint8_t *target, int64_t tlen,
                                         const uint8_t *query, int64_t qlen,
                                         const char *seed_pattern, int32_t input_codes,
                                         const sfe_hit *hits, int64_t nhits,
                                         const int32_t scores[16], int32_t X, int32_t hsp_thresh,
                                         sfe_hsp *hsps, int64_t cap, int64_t *nhsps,
                                         sfe_stats *stats, void *stream) {
    if (!nhsps || !scores) return SFE_EINVAL;
    if (tlen < 0 || qlen < 0 || nhits < 0 || cap < 0) return SFE_EINVAL;
    if (tlen > kMaxBases || qlen > kMaxBases || nhits > kMaxHits) return SFE_ELIMIT;
    if (X < 0 || X >= (1 << 30) || (input_codes != 0 && input_codes != 1)) return SFE_EINVAL;
    // the walk's packed windows hold 64 x score in int32: the same bound as
    // every other entry point
    for (int i = 0; i < 16; i++)
        if (scores[i] < -(1 << 20) || scores[i] > (1 << 20)) return SFE_EINVAL;
    SeedPattern pat;
    if (parse(seed_pattern, &pat) != SFE_OK) return SFE_EINVAL;
    if ((tlen > 0 && !on_device(target)) || (qlen > 0 && !on_device(query)) ||
        (nhits > 0 && !on_device(hits)) || (cap > 0 && !on_device(hsps)))
        return SFE_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    SCK(cudaGetDevice(&dev));
    unsigned char *base = nullptr;
    const int r0 = scratch_address(dev, &base);
    if (r0 != SFE_OK) return r0;

    StaticSmall *small = reinterpret_cast<StaticSmall *>(base + kOffSmall);
    uint32_t *Tp = reinterpret_cast<uint32_t *>(base + kOffT) + SEQ_PAD;
    uint32_t *Qp = reinterpret_cast<uint32_t *>(base + kOffQ) + SEQ_PAD;
    uint32_t *Qm = reinterpret_cast<uint32_t *>(base + kOffQm) + SEQ_PAD;
    uint64_t *ka = reinterpret_cast<uint64_t *>(base + kOffKeysA);
    uint64_t *kb = reinterpret_cast<uint64_t *>(base + kOffKeysB);
    uint4 *queue = reinterpret_cast<uint4 *>(base + kOffQueue);
    void *tmp = base + kOffTmp;
    if (radix_sort_temp_bytes(kMaxHits) > kTmpBytes || hsp_sort_temp_bytes(kMaxHits) > kTmpBytes)
        return SFE_ELIMIT;

    // the array keeps the previous call's contents: clear what must start at zero
    SCK(cudaMemsetAsync(small, 0, sizeof(StaticSmall), st));
    SCK(cudaMemcpyAsync(small->scores, scores, 64, cudaMemcpyHostToDevice, st));
    SCK(launch_pack(target, tlen, input_codes, Tp, &small->status, st));
    SCK(launch_pack(query, qlen, input_codes, Qp, &small->status, st));
    SCK(launch_revcomp(Qp, qlen, Qm, st));
    SCK(launch_public_to_walk(hits, nhits, tlen, qlen, pat.span, ka, &small->status, st));
    // (strand, diagonal, t): three stable passes, least significant first
    uint64_t *cur = ka, *oth = kb;
    bool in_b = false;
    SCK(radix_sort(cur, oth, nullptr, nullptr, nhits, 0, bits_of(tlen), tmp, &in_b,
                   &small->status, st));
    if (in_b) std::swap(cur, oth);
    SCK(radix_sort(cur, oth, nullptr, nullptr, nhits, 32, 32 + bits_of(tlen + qlen), tmp, &in_b,
                   &small->status, st));
    if (in_b) std::swap(cur, oth);
    SCK(radix_sort(cur, oth, nullptr, nullptr, nhits, 63, 64, tmp, &in_b, &small->status, st));
    if (in_b) std::swap(cur, oth);
    if (nhits > 0) {
        g_launches++;
        static_split_kernel<<<1, 1, 0, st>>>(cur, nhits, &small->split);
        SCK(cudaGetLastError());
    }
    StaticSmall hs;
    SCK(cudaMemcpyAsync(&hs, small, sizeof(hs), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    int r = device_status(hs.status);
    if (r != SFE_OK) return r;
    const long long split = nhits > 0 ? (long long)hs.split : 0;

    WalkParams wp{};
    wp.T = Tp;
    wp.tlen = tlen;
    wp.qlen = qlen;
    wp.span = pat.span;
    wp.xdrop = X;
    wp.thresh = hsp_thresh;
    wp.flags = 0;
    wp.lane_cap = DEFAULT_LANE_CAP;
    wp.qoff = qlen - pat.span;
    wp.scores = small->scores;
    wp.Ecarry = nullptr;
    wp.hsps = reinterpret_cast<Hsp *>(hsps);  // written in place, sorted below
    wp.hsp_cap = (unsigned long long)cap;
    wp.ctr = &small->ctr;
    wp.queue = queue;
    wp.queue_cap = (unsigned long long)kMaxHits;
    wp.queue_len = &small->queue_len;
    for (int s = 0; s < 2; s++) {
        const long long b = s ? split : 0, e = s ? nhits : split;
        if (e <= b) continue;
        wp.strand = s;
        wp.Q = s ? Qm : Qp;
        SCK(cudaMemsetAsync(&small->queue_len, 0, 4, st));
        SCK(launch_walk_lanes(cur + b, e - b, wp, 0, st));
        SCK(launch_walk_warps(cur + b, e - b, wp, 0, st));
    }
    SCK(cudaMemcpyAsync(&hs, small, sizeof(hs), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    r = device_status(hs.ctr.status);
    if (r != SFE_OK) return r;
    *nhsps = (int64_t)hs.ctr.hsps;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->hits = nhits;
        stats->extended = (int64_t)hs.ctr.extended;
        stats->cells = (int64_t)hs.ctr.cells;
        stats->hsps = (int64_t)hs.ctr.hsps;
        stats->lane_tasks = (int64_t)hs.ctr.lane_tasks;
        stats->warp_tasks = (int64_t)hs.ctr.warp_tasks;
        stats->warp_cells = (int64_t)hs.ctr.warp_cells;
        stats->shadow_cells = (int64_t)hs.ctr.shadow;
        stats->tiles = 1;
    }
    if ((long long)hs.ctr.hsps > cap) return SFE_EOVERFLOW;
    if (hs.ctr.hsps > 1) {
        SCK(hsp_sort(reinterpret_cast<Hsp *>(hsps), (long long)hs.ctr.hsps, bits_of(tlen),
                     bits_of(qlen), tmp, &small->status, st));
        SCK(cudaMemcpyAsync(&hs, small, sizeof(hs), cudaMemcpyDeviceToHost, st));
        SCK(cudaStreamSynchronize(st));
        r = device_status(hs.status);
        if (r != SFE_OK) return r;
    }
    return SFE_OK;
}
