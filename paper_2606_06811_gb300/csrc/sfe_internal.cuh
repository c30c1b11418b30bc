// Internal declarations shared by the CUDA translation units of libsfe.
//
// Packed sequence layout (every kernel that reads bases uses it):
//   2 bits per base, 16 bases per uint32, base i in word i/16 at bits 2*(i%16).
//   A packed buffer holds SEQ_PAD words of zeros before base 0 and SEQ_PAD
//   words after the last base, so a 16- or 32-base window that starts up to
//   64 bases before 0 or ends up to 64 bases past the end stays in bounds.
//   Kernels receive a pointer to the word that holds base 0.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "sfe.h"

namespace sfe {

constexpr int SEQ_PAD = 4;          // words of padding on each side
constexpr int MAX_SPAN = 32;
constexpr int MAX_WEIGHT = 14;      // 4^14 + 1 offsets = 1 GiB of CSR
constexpr int BLOCK = 256;
// Bases per side a lane scores before it hands its diagonal to the warp tier
// (the default of sfe_params.lane_cap; a sweep on the 10 Mb pair: 128, 256,
// 512 and 1024 give 10.12, 9.98, 10.40 and 10.41 ms of walk).
constexpr int DEFAULT_LANE_CAP = 256;

// Device status bits (accumulated with atomicOr into one uint32).
constexpr uint32_t ST_BAD_SYMBOL = 1u;
constexpr uint32_t ST_SCORE_OVERFLOW = 2u;
constexpr uint32_t ST_HSP_OVERFLOW = 4u;
constexpr uint32_t ST_QUEUE_OVERFLOW = 8u;
constexpr uint32_t ST_BAD_HIT = 16u;
constexpr uint32_t ST_TIMEOUT = 32u;  // a bounded device wait ran out

struct SeedPattern {
    int span;
    int weight;
    int care[MAX_SPAN];
    int step;  // index stride: only target positions t with t % step == 0 are seeds
};

// Target positions a pattern indexes in a sequence of n bases: every step-th
// of the n - span + 1 positions, from 0.
__host__ __device__ inline long long indexed_positions(const SeedPattern &pat, long long n) {
    const long long npos = n - pat.span + 1;
    return npos > 0 ? (npos + pat.step - 1) / pat.step : 0;
}

// Counters written by the walkers (one struct in device memory).
struct DevCounters {
    unsigned long long extended;
    unsigned long long cells;
    unsigned long long hsps;       // HSPs found (may exceed the HSP buffer)
    unsigned long long lane_tasks;
    unsigned long long warp_tasks; // queue entries
    unsigned long long warp_cells; // cells scored by the warp tier
    unsigned long long ext_logged; // extensions selected for the extension log
    unsigned long long shadow;     // lane cells of extensions handed to the warp tier
    unsigned long long deferred;   // hand-off entries left to the follow-up warp launch
    unsigned int status;
    unsigned int pad;
};

// HSP as written by the walkers (same layout as sfe_hsp).
struct Hsp {
    int32_t strand, tpos, qpos, len, score;
};

// HSP of a batch of pairs (same layout as sfe_batch_hsp).
struct BatchHsp {
    int32_t pair, strand, tpos, qpos, len, score;
};

// One pair of a batch: where its sequences sit in the concatenated packed
// buffers and where its seeding buckets sit in the batch index.
struct PairInfo {
    long long toff;     // first base of the target in the packed targets
    long long qoff;     // first base of the query in the packed queries
    long long qoff_rc;  // first base of its reverse complement in the packed rc buffer
    long long boff;     // first bucket of its index
    int tlen, qlen;
    int bbits;          // its index has 2^bbits buckets (top bits of the seed key)
    int pad;
};

// A hit in the walk layout: high word = diagonal index D = t - q + (qlen - span),
// low word = t. Sorting by the high word (stably, from query order) groups a
// diagonal's hits in increasing t.
__host__ __device__ inline uint64_t make_hit(uint32_t D, uint32_t t) {
    return ((uint64_t)D << 32) | t;
}

// 16 bases starting at base p (p may be negative down to -64): base p in bits 0-1.
__device__ __forceinline__ uint32_t win16(const uint32_t *__restrict__ S, long long p) {
    long long w = p >> 4;  // arithmetic shift: floor division
    uint32_t lo = __ldg(S + w), hi = __ldg(S + w + 1);
    return __funnelshift_r(lo, hi, (uint32_t)(p & 15) * 2u);
}

__device__ __forceinline__ uint32_t base_at(const uint32_t *__restrict__ S, long long p) {
    return (__ldg(S + (p >> 4)) >> ((uint32_t)(p & 15) * 2u)) & 3u;
}

// ------------------------------------------------------------ host launchers
// All launchers queue work on `st` and return cudaGetLastError().

// Kernels launched by this library from the calling host thread since it was
// loaded (incremented at every launch site). Thread-local: a context is used
// by one host thread at a time, so a call's launch count is this counter's
// change across the call, whatever other threads launch meanwhile.
extern thread_local unsigned long long g_launches;

// Streaming-multiprocessor count of the current device (looked up once per
// device; grids of persistent and strided kernels are sized from it).
int device_sms();

// Runs set() (a cudaFuncSetAttribute, which holds per device) the first time
// it is reached on the current device; `done` keeps one bit per device.
// Two threads may both run set() once: it is idempotent.
template <class F>
cudaError_t once_per_device(std::atomic<unsigned long long> &done, F set) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = set();
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// bytes -> packed words (n bases). codes: 0 = ASCII, 1 = 2-bit codes.
// dst points at the word of base 0 of a buffer with SEQ_PAD words on each side;
// the padding is zeroed too. Bad symbols set ST_BAD_SYMBOL in *status.
cudaError_t launch_pack(const uint8_t *src, long long n, int codes, uint32_t *dst,
                        uint32_t *status, cudaStream_t st);
// Reverse complement of a packed sequence of n bases into another padded buffer.
cudaError_t launch_revcomp(const uint32_t *src, long long n, uint32_t *dst, cudaStream_t st);
// cell plane (4 bits per base, PLANE_PAD zero words on each side) of a packed
// sequence: plane_words is the allocation, dst the base 0 pointer
constexpr int PLANE_PAD = 4;
size_t plane_words(long long n);
cudaError_t launch_plane(const uint32_t *S, long long n, int shift, uint32_t *dst, cudaStream_t st);
// keys[j] = (seed key of p) << 32 | p for p = j * step, j < indexed_positions(pat, n).
cudaError_t launch_seed_keys(const uint32_t *S, long long n, SeedPattern pat, uint64_t *keys,
                             cudaStream_t st);
// CSR bucket sizes (counts zeroed by the caller) and the positions column from
// keys sorted by their high word; offsets = exclusive scan of counts. With
// shift > 0 (a sparse index) the buckets are the keys' top bits (key >> shift)
// and low[i] receives the remaining bits of entry i's key.
cudaError_t launch_csr_counts(const uint64_t *sorted, long long m, uint32_t *counts,
                              uint32_t *positions, int shift, uint16_t *low, cudaStream_t st);

// Stable LSD radix sort of n (< 2^32) uint64 keys by bits [lo, hi), optional
// uint32 values carried along. Uses (a, b) ping-pong and returns in
// *result_in_b whether the sorted data ended in the b buffers.
// tmp: radix_sort_temp_bytes(n). `status` receives device error bits.
size_t radix_sort_temp_bytes(long long n);
cudaError_t radix_sort(uint64_t *keys_a, uint64_t *keys_b, uint32_t *vals_a, uint32_t *vals_b,
                       long long n, int lo, int hi, void *tmp, bool *result_in_b, uint32_t *status,
                       cudaStream_t st);
// The same with the key count in device memory (*nd, at most n): the grid is
// sized for n and each kernel reads the count, so no host synchronisation is
// needed (the form a captured CUDA graph replays).
cudaError_t radix_sort_dev(uint64_t *keys_a, uint64_t *keys_b, uint32_t *vals_a, uint32_t *vals_b,
                           long long n, const unsigned long long *nd, int lo, int hi, void *tmp,
                           bool *result_in_b, uint32_t *status, cudaStream_t st);

// Exclusive scan of n uint32 into uint64 (out has n + 1 entries: out[n] = total).
size_t scan_temp_bytes(long long n);
cudaError_t scan_u32_to_u64(const uint32_t *in, unsigned long long *out, long long n, void *tmp,
                            cudaStream_t st);
cudaError_t scan_u32_to_u32(const uint32_t *in, uint32_t *out, long long n, void *tmp,
                            cudaStream_t st);

// Seed-hit counting and writing for query positions [q0, q1) of one strand.
struct HitParams {
    SeedPattern pat;
    int transition;
    long long qlen;
    long long qoff;  // qlen - span, so D = t - q + qoff >= 0
    // sparse index (low != nullptr): CSR over key >> shift, low[j] = the
    // entry's key & (2^shift - 1); a probe scans its bucket for its low bits
    int shift;
    const uint16_t *low;
};
// ncount[k]: hits of key k's probe set (launch_neighbor_counts), or null to
// count by probing the offsets.
cudaError_t launch_neighbor_counts(const uint32_t *offsets, const SeedPattern &pat,
                                   int transition, uint32_t *ncount, cudaStream_t st);
cudaError_t launch_hit_count(const uint32_t *Qs, HitParams hp, const uint32_t *offsets,
                             const uint32_t *ncount, long long q0, long long q1, uint32_t *counts,
                             cudaStream_t st);
// Merged probe-set lists (off2: exclusive scan of the probe-set sizes, 4^weight
// + 1 entries; pos2: their positions back to back).
cudaError_t launch_merged_fill(const uint32_t *offsets, const uint32_t *positions,
                               const SeedPattern &pat, int transition, const uint32_t *off2,
                               uint32_t *pos2, cudaStream_t st);
// nhits: the hits of [q0, q1) (picks a per-thread or a per-warp writer);
// off2 / pos2: merged lists, or null to read the probes' buckets
cudaError_t launch_hit_write(const uint32_t *Qs, HitParams hp, const uint32_t *offsets,
                             const uint32_t *positions, const uint32_t *off2,
                             const uint32_t *pos2, long long q0, long long q1,
                             const unsigned long long *starts, unsigned long long base,
                             unsigned long long nhits, uint64_t *hits, cudaStream_t st);

struct WalkParams {
    const uint32_t *T;   // packed target (base 0)
    const uint32_t *Q;   // packed query strand (base 0)
    // cell planes of the target and of the query strand (4 bits per base,
    // base 0 pointers; one pair only, nullptr: the walk reads T and Q)
    const uint32_t *TN, *QN;
    long long tlen, qlen;
    int span;
    int strand;
    int xdrop;
    int thresh;
    int flags;
    int lane_cap;
    long long qoff;      // qlen - span
    const int32_t *scores;  // 16 int32 in device memory
    int32_t *Ecarry;     // per-diagonal E carried across query tiles (nullptr: single tile)
    Hsp *hsps;
    unsigned long long hsp_cap;
    DevCounters *ctr;
    uint4 *queue;        // hand-off queue: (hit index, E, unused, unused)
    unsigned long long queue_cap;
    unsigned int *queue_len;
    // batch of pairs (pairs == nullptr for a single pair): the hit word is
    // pair << (dbits + 1) | strand << dbits | local diagonal
    const PairInfo *pairs;
    const uint32_t *Qrc;  // packed reverse complements of the queries
    int dbits;
    BatchHsp *bhsps;
    // persistent walk: lanes take chunks of `chunk` hits from a work counter
    // (in `order` when given), and warps out of lane work consume the hand-off
    // queue in the same launch; queue entries of this call carry `epoch`
    unsigned int *work_next;
    unsigned int *warps_done;
    unsigned int *queue_take;
    const uint32_t *order;
    uint32_t nchunks, chunk, epoch;
    // hit count in device memory (at most the launch's n), for launches that
    // must not wait for the host (graph replay); null: the launch's n
    const unsigned long long *nd;
    long long spin_limit;  // polls of a hand-off entry before its consumer leaves it (and the
                           // rest of the queue) to the follow-up warp launch
    int phantom;           // test hook: reserve one queue slot that is never written
    // follow-up warp launch after a persistent walk: only entries published by
    // this call (z == epoch) that no consumer finished (w != epoch)
    int deferred_only;
    // sampled log of extensions (elog == nullptr: none)
    sfe_ext_record *elog;
    unsigned long long elog_cap;
    uint32_t elog_every;
};

// Whether the extension of hit (pair, strand, t, q) goes to the log: a hash of
// the hit, so the sample does not depend on the order of the walk.
__device__ __forceinline__ bool ext_sampled(uint32_t every, int pair, int strand, long long t,
                                            long long q) {
    uint32_t h = (uint32_t)t * 0x9E3779B1u ^ (uint32_t)q * 0x85EBCA77u ^
                 (uint32_t)pair * 0xC2B2AE3Du ^ (uint32_t)strand * 0x27D4EB2Fu;
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    h *= 0x846CA68Bu;
    h ^= h >> 16;
    return h % every == 0;
}
// Walks of hits sorted by (diagonal word, t): lanes own contiguous hit ranges
// (lanes_per_sm sizes the ranges; 0 = default); warps finish the diagonals
// the lanes handed off.
cudaError_t launch_walk_lanes(const uint64_t *hits, long long n, WalkParams wp, int lanes_per_sm,
                              cudaStream_t st);
cudaError_t launch_walk_warps(const uint64_t *hits, long long n, WalkParams wp, int grid_warps,
                              cudaStream_t st);
// Chunk order of the persistent walk for a schedule (SFE_SCHED_*): *order is
// left null for the natural order. tmp: walk_schedule_temp_bytes(n, chunk).
// SFE_SCHED_PREDICTED ranks chunks with the work predictor `model`.
size_t walk_schedule_temp_bytes(long long n, uint32_t chunk);
// Hits per chunk of the persistent walk when the caller leaves it to the
// library: about 16 chunks per resident lane, 16 to 256 hits.
uint32_t walk_auto_chunk(long long n);
cudaError_t launch_walk_schedule(const uint64_t *hits, long long n, const WalkParams &wp,
                                 int schedule, const void *model, void *tmp, uint32_t **order,
                                 uint32_t *status, cudaStream_t st);

// Work predictor (MLP, see mlp.cu): parameter count, inference blob size,
// initialisation, FP16 packing, loss/gradient/prediction over extension
// records, Adam, and the per-chunk predicted work used by the schedule.
int mlp_param_count();
size_t mlp_model_bytes();
cudaError_t launch_mlp_init(float *P, unsigned long long seed, cudaStream_t st);
cudaError_t launch_mlp_pack(const float *P, void *model, cudaStream_t st);
cudaError_t launch_mlp_fwd_bwd(const uint32_t *T, long long tlen, const uint32_t *Q,
                               const uint32_t *Qrc, long long qlen, const PairInfo *pairs,
                               int span, const sfe_ext_record *recs, const uint32_t *perm,
                               long long n, const float *P, float *grad, float *preds,
                               double *loss, cudaStream_t st);
cudaError_t launch_adam(float *P, const float *g, float *m, float *v, float lr, int step,
                        cudaStream_t st);
cudaError_t launch_mlp_predict16(const uint32_t *T, long long tlen, const uint32_t *Q,
                                 const uint32_t *Qrc, long long qlen, const PairInfo *pairs,
                                 int span, const sfe_ext_record *recs, long long n,
                                 const void *model, float *preds, cudaStream_t st);
cudaError_t launch_validate_records(const sfe_ext_record *recs, long long n, int npairs,
                                    uint32_t *status, cudaStream_t st);
// A permutation of 0..n-1 from (seed, epoch): random keys sorted on the device.
cudaError_t launch_perm(long long n, unsigned long long seed, int epoch, uint64_t *ka,
                        uint64_t *kb, void *tmp, uint32_t *perm, uint32_t *status,
                        cudaStream_t st);
cudaError_t launch_chunk_predict(const uint64_t *hits, long long n, uint32_t chunk,
                                 uint32_t nchunks, const WalkParams &wp, const void *model,
                                 uint64_t *keys, cudaStream_t st);
// The speculative window walk (one warp per diagonal, `window` hits of it
// extended at once and committed in t order; window = 1, 2, 4, ..., 32):
// wp.work_next zeroed by the caller; one pair or hit list (no wp.pairs).
cudaError_t launch_walk_speculative(const uint64_t *hits, long long n, WalkParams wp, int window,
                                    cudaStream_t st);
// Both tiers in one persistent launch fed by the work counter and the queue
// (wp.work_next, warps_done, queue_take, queue_len zeroed by the caller).
cudaError_t launch_walk_persistent(const uint64_t *hits, long long n, WalkParams wp,
                                   cudaStream_t st);

// Gapped Y-drop extension (ydrop.cu): one warp per anchor half. anchors[k] =
// (strand, t, q, unused); task 2k is anchor k's forward half (T[t..],
// Qs[q..]), task 2k + 1 its backward half (T[..t), Qs[..q) reversed); Qs is
// the packed query (strand 0) or its reverse complement (strand 1).
constexpr int YD_MAX_BAND = 256;
struct YdParams {
    int32_t scores[16];
    int32_t gap_open, gap_extend, ydrop;
    int32_t band;  // cells per anti-diagonal, 1..YD_MAX_BAND
};
struct YdHalf {
    int32_t best, bi, bj;  // best score, bases of T and Q consumed at the first best cell
    uint32_t status;       // ST_SCORE_OVERFLOW
    long long cells;       // DP cells computed beyond the origin
};
size_t ydrop_smem_bytes(int band);
cudaError_t launch_ydrop(const uint32_t *T, long long tlen, const uint32_t *Qp,
                         const uint32_t *Qm, long long qlen, const int4 *anchors, int nanchors,
                         const YdParams &prm, YdHalf *out, cudaStream_t st);

// Sort HSPs in place by (strand, tpos, qpos, len, score); tpos < 2^tbits,
// qpos < 2^qbits, tbits + qbits <= 62. tmp: hsp_sort_temp_bytes(n).
size_t hsp_sort_temp_bytes(long long n);
cudaError_t hsp_sort(Hsp *hsps, long long n, int tbits, int qbits, void *tmp, uint32_t *status,
                     cudaStream_t st);

// Batch of pairs: per-pair hashed seeding index (cnt and off hold nbuckets and
// nbuckets + 1 entries, entries one per target seed position), per-pair hit
// count and write over (strand, query position), and the HSP order (pair,
// strand, tpos, qpos, len, score) with pairs < 2^pbits, positions < 2^lbits.
// Work items are chunks of batch_item_size() positions of one pair, numbered
// pair by pair: tprefix / qprefix (npairs + 1 entries, device) give each pair's
// first item; query items hold both strands of a chunk next to each other.
int batch_item_size();
// The two split-key tables of every pair (see batch.cu): nbuckets per table,
// cnt 2 * nbuckets, off 2 * nbuckets + 1, entries two per target position,
// slots one per target base (scratch). PairInfo.bbits must be at most
// batch_table_bits(weight).
int batch_table_bits(int weight);
cudaError_t launch_batch_index(const uint32_t *T, const PairInfo *pairs, const long long *tprefix,
                               long long titems, int npairs, SeedPattern pat, uint32_t *cnt,
                               long long nbuckets, uint32_t *off, uint64_t *entries, uint2 *slots,
                               void *tmp, cudaStream_t st);
// One pass: hits in no particular order, at most cap written, *total = all.
cudaError_t launch_batch_hit_emit(const uint32_t *Q, const uint32_t *Qrc, const PairInfo *pairs,
                                  const long long *qprefix, long long qitems, int npairs,
                                  int strands_mask, SeedPattern pat, int transition, int dbits,
                                  long long nbuckets, const uint32_t *off,
                                  const uint64_t *entries, unsigned long long *total,
                                  unsigned long long cap, uint64_t *hits, cudaStream_t st);
// Sort of a batch's HSPs by (pair, strand, tpos, qpos, len, score); n is the
// count, or with `nd` the capacity and *nd the count. *out receives the
// sorted array (in tmp, or h itself for n <= 1).
size_t batch_hsp_sort_temp_bytes(long long n);
cudaError_t batch_hsp_sort(BatchHsp *h, long long n, const unsigned long long *nd, int pbits,
                           int lbits, void *tmp, BatchHsp **out, uint32_t *status,
                           cudaStream_t st);

// Conversions between the public hit record and the walk layout.
cudaError_t launch_hits_to_public(const uint64_t *hits, long long n, int strand, long long qoff,
                                  sfe_hit *out, cudaStream_t st);
cudaError_t launch_public_to_walk(const sfe_hit *in, long long n, long long tlen, long long qlen,
                                  int span, uint64_t *out, uint32_t *status, cudaStream_t st);

}  // namespace sfe
