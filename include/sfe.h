/*
 * sfe.h - C ABI of the GB300 seed-filter-extend filter stage.
 *
 * The library computes the filter stage of the seed-filter-extend pipeline
 * (Section 1 of "Dependencies and Dataflow in Seed-Filter-Extend Pipelines"):
 * spaced-seed hits between a target T and both strands of a query Q
 * (12-of-19 seed 1110100110010101111 with transition tolerance, Section 2 and
 * Section 7), the loop-carried skip of hits that fall inside a region already
 * extended on their diagonal (Algorithm 1, the IsContained test and the
 * masking-list update), and the ungapped X-drop extension that turns the
 * surviving hits into HSPs (Section 2 and Section 8: a 1-D dynamic program
 * with no gaps). Every step runs in hand-written CUDA kernels for sm_103a.
 *
 * Conventions shared by every call:
 *  - Bases: ASCII A/C/G/T (either case), or 2-bit codes A=0 C=1 G=2 T=3 one per
 *    byte when sfe_params.input_codes = 1. Any other symbol gives SFE_EINVAL.
 *  - Coordinates are 0-based, half-open. Strand 0 is the query as given;
 *    strand 1 is its reverse complement and its coordinates index the reverse
 *    complement (qpos 0 is the complement of the last query base).
 *  - A hit (strand, tpos, qpos) means the seed pattern matches at T[tpos..] and
 *    Q_strand[qpos..]. Its diagonal is tpos - qpos.
 *  - The X-drop rule: each side extends base by base; it stops right after the
 *    first base at which (running maximum - running sum) > X, or at the end of
 *    either sequence; the HSP ends where the maximum was first reached. The HSP
 *    always holds the whole seed span. Scores are int32 sums of
 *    scores[4 * target_base + query_base].
 *  - A hit is skipped when tpos < E, E being the exclusive end of the last
 *    extended HSP on its (strand, diagonal); E is advanced by every extension
 *    (or only by those reaching hsp_thresh with SFE_SKIP_PASSING_ONLY).
 *  - Pointers may be device pointers (from cudaMalloc or a PyTorch CUDA
 *    tensor) or host pointers (pageable or pinned); the library detects which
 *    with cudaPointerGetAttributes and copies host data in and out itself.
 *  - Work is queued on the context's stream. Every call returns after its
 *    results (counts, stats, host outputs) are complete.
 *  - Outputs are caller-owned buffers with a capacity; when the result does
 *    not fit, the call returns SFE_EOVERFLOW and sets the needed count.
 *  - Scratch memory is owned by the context (grown on demand, reused across
 *    calls, freed by sfe_ctx_destroy). A context is not thread-safe; use one
 *    context per host thread.
 *  - Return codes: SFE_OK (0) or a negative SFE_E* code; sfe_last_error()
 *    describes the most recent failure of the calling thread.
 */
#ifndef SFE_H
#define SFE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SFE_OK 0
#define SFE_EINVAL (-1)    /* bad argument or symbol */
#define SFE_ENOMEM (-2)    /* device allocation failed */
#define SFE_ECUDA (-3)     /* a CUDA call failed */
#define SFE_ETIMEOUT (-4)  /* a bounded device wait ran out (kept for the ABI; the persistent
                              walk now hands late entries to a follow-up launch instead) */
#define SFE_EOVERFLOW (-5) /* output capacity too small (needed count returned), or a score left int32 */
#define SFE_ELIMIT (-6)    /* input larger than the fixed scratch of sfe_ungapped_xdrop_static */

/* sfe_params.flags */
#define SFE_SKIP_PASSING_ONLY 1 /* advance E only for HSPs with score >= hsp_thresh */
#define SFE_TIME_STAGES 2       /* time each stage with CUDA events on the context's stream */
#define SFE_NO_CELL_PLANES 4    /* sfe_run: lane windows read the 2-bit words even where the
                                   4-bit cell planes of T and of each query strand (built
                                   when they take at most 64 MB) would fit; the output is the
                                   same either way */

/* Stages of a call, indexes of sfe_stats.stage_ms / stage_launches. */
enum {
    SFE_STAGE_PACK = 0,       /* 2-bit packing and reverse complement */
    SFE_STAGE_INDEX = 1,      /* spaced keys, radix sort, CSR table */
    SFE_STAGE_COUNT = 2,      /* hits per query position and their scan */
    SFE_STAGE_WRITE = 3,      /* hit records */
    SFE_STAGE_SORT = 4,       /* grouping of hits by diagonal */
    SFE_STAGE_SCHEDULE = 5,   /* order of the persistent walk's work chunks */
    SFE_STAGE_WALK_LANES = 6, /* skip + X-drop, one lane per diagonal */
    SFE_STAGE_WALK_WARPS = 7, /* skip + X-drop, one warp per handed-off diagonal */
    SFE_STAGE_OUTPUT = 8,     /* HSP sort and copy-out */
    SFE_NSTAGES = 9
};

typedef struct sfe_ctx sfe_ctx;
typedef struct sfe_index sfe_index;

/* One seed hit. */
typedef struct {
    int32_t strand, tpos, qpos;
} sfe_hit;

/* One HSP (high-scoring ungapped segment); len is the same in T and Q. */
typedef struct {
    int32_t strand, tpos, qpos, len, score;
} sfe_hsp;

/* One HSP of a batch of pairs. */
typedef struct {
    int32_t pair, strand, tpos, qpos, len, score;
} sfe_batch_hsp;

/* One logged extension (see sfe_params.ext_log): the seed hit and the bases
 * its X-drop scored on each side. Its work in cells is span + right + left. */
typedef struct {
    int32_t pair, strand, t, q, right, left;
} sfe_ext_record;

typedef struct {
    const char *seed_pattern; /* '1' care, '0' don't care; span <= 32, weight <= 14; NULL = 12of19 */
    int32_t transition;       /* 1: at most one care position may be a transition (A<->G, C<->T) */
    int32_t strands;          /* bit 0: strand 0 (plus), bit 1: strand 1 (minus) */
    int32_t scores[16];       /* scores[4 * target_base + query_base] */
    int32_t xdrop;            /* X >= 0 (and < 2^30) */
    int32_t hsp_thresh;       /* HSPs with score >= hsp_thresh are reported */
    int32_t flags;            /* SFE_SKIP_PASSING_ONLY, SFE_TIME_STAGES, SFE_NO_CELL_PLANES */
    int32_t input_codes;      /* 0: ASCII ACGTacgt, 1: codes 0..3 */
    int32_t lane_cap;         /* bases per side a lane extends before handing the diagonal to a warp; 0 = default */
    int32_t lanes_per_sm;     /* lane-tier threads per SM sharing a tile's hits (sizes their hit ranges); 0 = default */
    int64_t tile_hits;        /* hits per query tile (bounds scratch memory); 0 = default (2^30) */
    int32_t walk_chunk;       /* hits a lane takes per grab from the work counter; 0 = from the hit
                                 count (16 to 256, about 16 chunks per resident lane) */
    int32_t walk_mode;        /* SFE_WALK_PERSISTENT or SFE_WALK_TWO_LAUNCHES */
    int32_t walk_schedule;    /* order in which the persistent walk hands out chunks (SFE_SCHED_*);
                                 anything but SFE_SCHED_NATURAL needs SFE_WALK_PERSISTENT */
    int32_t ext_log_every;    /* log about 1 in ext_log_every extensions (0: no log) */
    sfe_ext_record *ext_log;  /* device buffer for the log; the choice of logged hits is a hash of
                                 (pair, strand, t, q), so it does not depend on the schedule */
    int64_t ext_log_cap;      /* records the buffer holds (further ones are counted, not written) */
    const void *model;        /* device weights of the work predictor (SFE_SCHED_PREDICTED) */
    int32_t wait_limit;       /* polls (at most about 1 us each) a warp of the persistent walk
                                 waits for a hand-off entry to be published before it leaves
                                 that entry and the rest of the queue to a follow-up warp
                                 launch on the same stream (the output is the same either way;
                                 see stats.deferred_tasks); 0 = default (2^20) */
    int32_t test_hooks;       /* SFE_TEST_* bits; 0 in normal use */
    int32_t step;             /* index stride (Section 7's spacing between seeds): only target
                                 positions t with t % step == 0 are indexed, so only they start
                                 hits; 0 or 1 = every position */
    int32_t spec_window;      /* SFE_WALK_SPECULATIVE: hits extended at once per diagonal, 1, 2,
                                 4, 8, 16 or 32; 0 = 8 */
} sfe_params;

/* sfe_params.test_hooks (no counterpart in the paper: they let tests drive the
 * library's recovery paths without faulting a GPU). SFE_TEST_UNPUBLISHED_QUEUE_ENTRY
 * reserves one slot of the persistent walk's hand-off queue that is never
 * written, as if its producer had not run yet: the warp that takes it waits
 * until wait_limit runs out and leaves the queue to the follow-up launch, which
 * skips the slot (it holds no task); the output is the oracle's all the same
 * and stats.deferred_tasks counts the warps that gave up. */
#define SFE_TEST_UNPUBLISHED_QUEUE_ENTRY 1
/* SFE_TEST_DENSE_INDEX builds the position table over all 4^weight keys (with
 * the per-key probe-set tables) even for a target that fills few of them,
 * where the library otherwise indexes the keys' top bits (a sparse index);
 * both give the same hits. */
#define SFE_TEST_DENSE_INDEX 2

/* sfe_params.walk_schedule: the order of work never changes the output, only
 * how evenly it spreads over the warps */
#define SFE_SCHED_NATURAL 0       /* chunks in hit order */
#define SFE_SCHED_LARGEST_FIRST 1 /* chunks starting in larger diagonals (more hits) first */
#define SFE_SCHED_PREDICTED 2     /* chunks with more predicted work first (model in params) */
#define SFE_SCHED_RANDOM 3        /* chunks in a fixed pseudo-random order (a control) */

/* sfe_params.walk_mode */
#define SFE_WALK_TWO_LAUNCHES 0 /* lanes own fixed hit ranges; a second launch drains the queue */
#define SFE_WALK_PERSISTENT 1   /* one launch: lanes pull chunks from a device counter, then
                                   the same warps drain the hand-off queue */
#define SFE_WALK_SPECULATIVE 2  /* Algorithm 3's speculative batch on the per-diagonal skip: a
                                   warp per diagonal extends the next spec_window hits not yet
                                   covered at once (32 / spec_window lanes each) and commits
                                   them in t order; hits an earlier commit covers are skipped
                                   and their work is counted in stats.shadow_cells. Same output
                                   as the other modes, for a pair, a hit list or a batch */

/* Statistics of one call. cells is the work measure of the method: seed span
 * plus the bases scored on both sides, summed over hits that were extended. */
typedef struct {
    int64_t hits;       /* seed hits enumerated */
    int64_t extended;   /* hits extended (not skipped) */
    int64_t cells;      /* span + bases scored, over extended hits */
    int64_t hsps;       /* HSPs with score >= hsp_thresh */
    int64_t lane_tasks; /* diagonals walked by single lanes */
    int64_t warp_tasks; /* diagonals handed to whole warps */
    int64_t warp_cells; /* cells scored by the warp tier (the rest by lanes) */
    int64_t tiles;      /* query tiles processed */
    int64_t launches;   /* kernels this call launched */
    int64_t ext_logged; /* extensions selected for the log (may exceed ext_log_cap) */
    int64_t shadow_cells; /* work not in cells: the cells a lane scored on an extension before it
                             handed the diagonal to the warp tier, which scores it again, or
                             (SFE_WALK_SPECULATIVE) the work on hits extended speculatively and
                             then found covered */
    double stage_ms[SFE_NSTAGES];        /* device time per stage (with SFE_TIME_STAGES) */
    int64_t stage_launches[SFE_NSTAGES]; /* kernels launched per stage (with SFE_TIME_STAGES) */
    int64_t deferred_tasks; /* persistent walk: warps that stopped waiting for a hand-off entry
                               and left the rest of the queue to the follow-up warp launch */
} sfe_stats;

/* Fill *p with the defaults: 12of19 with one transition, both strands,
 * HOXD70 scores, X = 910, hsp_thresh = 3000, the persistent walk with chunks
 * sized from the hit count. Returns SFE_OK. */
int sfe_params_default(sfe_params *p);

const char *sfe_strerror(int code);
const char *sfe_last_error(void);

/* Create a context on CUDA device `device` with its own non-blocking stream. */
int sfe_ctx_create(int device, sfe_ctx **out);
/* Queue later work on `stream` (a cudaStream_t, e.g. a PyTorch stream); NULL
 * restores the context's own stream. The caller keeps the stream alive. */
int sfe_ctx_set_stream(sfe_ctx *ctx, void *stream);
/* Walk settings for later sfe_ungapped_xdrop calls on this context (that call
 * takes the method's parameters explicitly and no sfe_params): walk_mode,
 * lane_cap, walk_chunk, spec_window and the SFE_TIME_STAGES bit of flags are
 * copied from *params; NULL restores the defaults of sfe_params_default. The
 * output never depends on them. SFE_EINVAL on settings check_params rejects. */
int sfe_ctx_set_walk(sfe_ctx *ctx, const sfe_params *params);
/* Test hook (no counterpart in the paper): the next n device allocations of
 * the context's scratch arena fail as if the device were out of memory, so
 * the calls that need them return SFE_ENOMEM. n = 0 clears it. */
int sfe_ctx_fail_next_allocs(sfe_ctx *ctx, int32_t n);
/* Test hook (no counterpart in the paper): the library's stable LSD radix
 * sort on n 64-bit keys in device memory, ordered by bits [lo, hi) (0 <= lo <
 * hi <= 64), in place; with device_count != 0 the count is first copied to
 * the device and the sort runs in the form a captured batch uses (grids for n,
 * count read on the device). Keys must be 16-byte aligned. */
int sfe_test_radix_sort(sfe_ctx *ctx, uint64_t *keys, int64_t n, int32_t lo, int32_t hi,
                        int32_t device_count);
void sfe_ctx_destroy(sfe_ctx *ctx);

/*
 * Seeding index over the target (the "position table" of Section 5):
 * 2-bit packing, spaced-seed keys at every target position, a stable device
 * radix sort by key and a CSR table of 4^weight + 1 offsets. target: tlen
 * bases, host or device. Only seed_pattern, transition and input_codes of
 * *params are used. The index keeps the packed target; free it with
 * sfe_index_free. SFE_EINVAL on a bad pattern or symbol.
 */
int sfe_index_build(sfe_ctx *ctx, const uint8_t *target, int64_t tlen, const sfe_params *params,
                    sfe_index **out);
void sfe_index_free(sfe_index *index);

/*
 * Seed hits of the query against the index (Section 2 and Section 7), for the
 * strands in the bit mask `strands`. hits: caller buffer of `cap` records (host
 * or device), written sorted by (strand, diagonal, tpos). *nhits receives the
 * number of hits; if it exceeds cap nothing is written and SFE_EOVERFLOW is
 * returned.
 */
int sfe_seed_hits(sfe_ctx *ctx, const sfe_index *index, const uint8_t *query, int64_t qlen,
                  int32_t strands, sfe_hit *hits, int64_t cap, int64_t *nhits);

/*
 * Per-diagonal skip and ungapped X-drop over a hit list (Algorithm 1 with the
 * X-drop filter, Section 2 and Section 8). hits: nhits records in any order
 * (host or device); each is grouped by (strand, diagonal) and walked in tpos
 * order. scores: 16 int32 as in sfe_params. hsps: caller buffer of cap
 * records (host or device), written sorted by (strand, tpos, qpos, len,
 * score). *nhsps receives the HSP count (SFE_EOVERFLOW if above cap). stats
 * may be NULL. A hit whose seed span leaves either sequence gives SFE_EINVAL.
 */
int sfe_ungapped_xdrop(sfe_ctx *ctx, const sfe_index *index, const uint8_t *query, int64_t qlen,
                       const sfe_hit *hits, int64_t nhits, const int32_t scores[16], int32_t X,
                       int32_t hsp_thresh, sfe_hsp *hsps, int64_t cap, int64_t *nhsps,
                       sfe_stats *stats);

/*
 * The whole filter stage for one pair: index, hits on the requested strands,
 * skip and X-drop, sorted HSPs. Inputs and outputs host or device; the query
 * is processed in tiles of at most params->tile_hits hits with the skip state
 * carried across tiles, so the result does not depend on the tiling. Scratch
 * (context-owned, reused by later calls): the index, two hit buffers per
 * tile, and, unless SFE_NO_CELL_PLANES, 4-bit copies of the target and the
 * query strands when they take at most 64 MB. Lengths: each sequence below
 * 2^31 - 1024 bases and the two together below 2^31 (a diagonal index has 31
 * bits; the same holds for sfe_seed_hits and sfe_ungapped_xdrop), else
 * SFE_EINVAL before any GPU work.
 */
int sfe_run(sfe_ctx *ctx, const uint8_t *target, int64_t tlen, const uint8_t *query, int64_t qlen,
            const sfe_params *params, sfe_hsp *hsps, int64_t cap, int64_t *nhsps,
            sfe_stats *stats);

/*
 * The filter stage over a batch of independent target/query pairs (the
 * uneven, independent tasks of Section 8's load-balancing discussion, run as
 * one batch). targets / queries: the pairs' sequences back to back (host or
 * device); toff / qoff: host arrays of npairs + 1 offsets into them (toff[0] =
 * qoff[0] = 0, non-decreasing). Each pair is seeded against its own index and
 * extended within its own bounds, exactly as sfe_run would do it alone.
 * hsps: cap records (host or device) sorted by (pair, strand, tpos, qpos,
 * len, score), coordinates local to the pair. Limits: npairs <= 65536, every
 * sequence shorter than 2^20 bases, at most 2^32 - 1 hits in the batch.
 */
int sfe_run_batch(sfe_ctx *ctx, const uint8_t *targets, const int64_t *toff,
                  const uint8_t *queries, const int64_t *qoff, int32_t npairs,
                  const sfe_params *params, sfe_batch_hsp *hsps, int64_t cap, int64_t *nhsps,
                  sfe_stats *stats);

/*
 * A batch captured as a CUDA graph (the batch of sfe_run_batch, replayed).
 *
 * sfe_run_batch keeps every count of its pipeline in device memory (the hit
 * sort, the walk and the HSP sort read them there), so its device work needs
 * no host synchronisation between stages. A plan fixes the pairs' lengths
 * (toff, qoff as in sfe_run_batch) and the parameters, allocates every buffer
 * the pipeline touches, and captures pack, index, hit emission, sort, walk
 * and HSP sort into one CUDA graph on the context's stream; each run copies
 * new sequences of those lengths into the plan and replays the graph. hit_cap
 * bounds the hits of one run (0: an estimate from the lengths); a run that
 * finds more hits, or more HSPs than the plan holds, grows the plan, captures
 * it again and replays once more, so the output never depends on the caps.
 * The parameters are copied, but pointers in them (ext_log, model) are
 * captured as they are and must stay valid while the plan is used;
 * SFE_TIME_STAGES is rejected. A plan belongs to its context and its stream
 * and is not thread-safe.
 */
typedef struct sfe_batch_plan sfe_batch_plan;

int sfe_batch_plan_create(sfe_ctx *ctx, const int64_t *toff, const int64_t *qoff, int32_t npairs,
                          const sfe_params *params, int64_t hit_cap, sfe_batch_plan **out);
/* targets / queries: toff[npairs] / qoff[npairs] bases (host or device);
 * hsps, cap, nhsps and stats as in sfe_run_batch. */
int sfe_batch_plan_run(sfe_batch_plan *plan, const uint8_t *targets, const uint8_t *queries,
                       sfe_batch_hsp *hsps, int64_t cap, int64_t *nhsps, sfe_stats *stats);
void sfe_batch_plan_free(sfe_batch_plan *plan);

/*
 * Work predictor of the learned schedule (SFE_SCHED_PREDICTED).
 *
 * The paper names the load imbalance of X-drop extensions (Section 8: some
 * extensions run far longer than the median, and a warp waits for its
 * slowest lane) but learns nothing; this predictor is an addition that only
 * reorders independent work, so the HSP output never depends on it.
 *
 * Network: for a seed hit at (t, q) with seed span s, the 32 diagonal columns
 * left of the seed (T[t - 32 + i] against Q[q - 32 + i]) and the 32 right of
 * it (T[t + s + i] against Q[q + s + i]), i = 0..31, each one-hot over its
 * substitution class T xor Q of the 2-bit codes (0 match, 2 transition, 1 and
 * 3 transversions): input (column * 4 + class), columns 0..31 left and 32..63
 * right; a column outside either sequence is all zero. 256 inputs, two ReLU
 * layers of 64 and one linear output, the prediction of log(1 + right + left)
 * of the hit's extension (sfe_ext_record). Parameters:
 * sfe_mlp_param_count() FP32 values, in the order W1[256][64], b1[64],
 * W2[64][64], b2[64], W3[64], b3 (row = input unit). Training runs on the
 * device in FP32 with the library's own forward and backward kernels and
 * Adam; inference reads a model blob of sfe_mlp_model_bytes() bytes made by
 * sfe_mlp_pack (FP16 weights, FP32 biases, FP32 accumulation).
 */
typedef struct sfe_mlp_data sfe_mlp_data;

int32_t sfe_mlp_param_count(void);
int64_t sfe_mlp_model_bytes(void);

/* Random initial parameters (uniform, scaled by fan-in; b3 = 3) from `seed`
 * into the device buffer params. */
int sfe_mlp_init(sfe_ctx *ctx, float *params, uint64_t seed);

/* FP16 inference blob of the FP32 parameters; both device buffers. */
int sfe_mlp_pack(sfe_ctx *ctx, const float *params, void *model);

/*
 * Training samples: the extension records `recs` (n of them, host or device,
 * as logged by sfe_run with pair = 0 or by sfe_run_batch) and the sequences
 * they refer to, given as in sfe_run_batch (npairs = 1 with toff = {0, tlen},
 * qoff = {0, qlen} for sfe_run's records); span is the seed span of the run
 * that logged them (19 for the default pattern). The sequences are packed and
 * the records copied once; the handle owns its device memory. SFE_EINVAL when
 * a record's pair or strand is out of range (positions need no check: columns
 * outside a sequence are zero inputs).
 */
int sfe_mlp_data_create(sfe_ctx *ctx, const uint8_t *targets, const int64_t *toff,
                        const uint8_t *queries, const int64_t *qoff, int32_t npairs,
                        int32_t input_codes, int32_t span, const sfe_ext_record *recs, int64_t n,
                        sfe_mlp_data **out);
void sfe_mlp_data_free(sfe_mlp_data *data);

/*
 * Loss and gradient of the FP32 network over all samples: *loss (host)
 * receives the mean squared error of the prediction against
 * log(1 + right + left); grad (device, param_count floats, may be NULL)
 * receives the gradient of that mean; preds (device, n floats, may be NULL)
 * the predictions in record order.
 */
int sfe_mlp_loss_grad(sfe_ctx *ctx, const sfe_mlp_data *data, const float *params, float *grad,
                      float *preds, double *loss);

/*
 * Predictions of the FP16 inference model (sfe_mlp_pack) for every sample,
 * into preds (device, n floats) in record order. They run on the tensor cores
 * (FP16 inputs, FP32 accumulation), so the first layer's hidden units are
 * rounded to FP16 before the second layer.
 */
int sfe_mlp_predict(sfe_ctx *ctx, const sfe_mlp_data *data, const void *model, float *preds);

/*
 * Adam on minibatches: `epochs` passes, each over a fresh permutation of the
 * samples drawn from (seed, epoch), in minibatches of `batch` samples (the
 * last one smaller), learning rate lr, beta1 0.9, beta2 0.999, eps 1e-8.
 * params (device) is updated in place; the optimiser state starts at zero.
 * epoch_loss (host, `epochs` entries, may be NULL) receives each epoch's mean
 * squared error over its samples, each taken before its minibatch's update.
 */
int sfe_mlp_train(sfe_ctx *ctx, const sfe_mlp_data *data, float *params, int32_t epochs,
                  int32_t batch, float lr, uint64_t seed, double *epoch_loss);

/*
 * Gapped extension after the filter (the stage Algorithm 1 runs on the
 * filter's survivors: YDropExtension with containment skipping, and
 * Algorithm 3's speculative batches with a serial commit).
 *
 * Anchors: the midpoint (tpos + len/2, qpos + len/2) of each HSP (hsps:
 * nhsps records, host or device, as sfe_run writes them; the score orders
 * them), taken in decreasing HSP score (then strand, tpos, qpos, len). An
 * anchor that lies inside the box [tstart, tend) x [qstart, qend) of an
 * alignment committed on its strand is skipped; the others are extended and
 * committed when their score reaches gapped_thresh.
 *
 * Extension: from the anchor forward and backward, the affine-gap dynamic
 * program (substitutions scores[4 * target_base + query_base], a gap of L
 * bases costs gap_open + L * gap_extend) by anti-diagonals: a cell is live
 * while its score is at least best - ydrop (best over the earlier
 * anti-diagonals); an anti-diagonal computes every cell from the lowest to
 * the highest that has a live neighbour on the previous one or a live
 * diagonal predecessor on the one before, at most `band` cells; a half stops
 * after two anti-diagonals without a live cell. Alignment score = the two
 * halves' best scores; its box runs from the backward half's best cell to the
 * forward half's (the first cell, by anti-diagonal then target offset, that
 * reached the best). One GPU warp per anchor half.
 *
 * Batches (Algorithm 3): the host takes the next `batch` anchors not
 * contained in what is committed (0: every anchor in one batch), the GPU
 * extends them all, and the host commits them in order, dropping those that
 * an alignment committed before them in the batch now contains (their work
 * is stats.shadow / shadow_cells). The output does not depend on the batch
 * size. Strand 1 coordinates index the reverse complement of the query.
 *
 * out: cap records (host or device), sorted by (strand, tstart, qstart,
 * tend, qend, score); *nout the count (SFE_EOVERFLOW if above cap, or if a
 * score left the int32 range). Limits: |scores| <= 2^15, gap costs and ydrop
 * in [0, 2^28], band 1..256.
 */
typedef struct {
    int32_t strand, tstart, tend, qstart, qend, score;
} sfe_galign;

typedef struct {
    int32_t scores[16];
    int32_t gap_open;      /* default 400 */
    int32_t gap_extend;    /* default 30 */
    int32_t ydrop;         /* default 9400 */
    int32_t gapped_thresh; /* default 3000 */
    int32_t band;          /* cells per anti-diagonal, 1..256; 0 = 256 */
    int32_t input_codes;   /* 0: ASCII ACGTacgt, 1: codes 0..3 */
    int64_t batch;         /* anchors per speculative batch; 0 = all in one batch */
} sfe_ydrop_params;

typedef struct {
    int64_t anchors;      /* HSPs given */
    int64_t skipped;      /* anchors contained when the scan reached them (never extended) */
    int64_t extended;     /* extensions whose result counts */
    int64_t cells;        /* DP cells of those extensions */
    int64_t shadow;       /* speculative extensions dropped at the commit */
    int64_t shadow_cells; /* their DP cells */
    int64_t committed;    /* alignments reported */
    int64_t batches;
    double device_ms;     /* extension kernels (CUDA events on the context's stream) */
    double total_ms;      /* the whole call, host scan and commit included (host clock) */
} sfe_ydrop_stats;

/* Fill *p with the defaults (HOXD70, 400/30, Y 9400, threshold 3000, band 256,
 * one batch). */
int sfe_ydrop_params_default(sfe_ydrop_params *p);
int sfe_gapped_extend(sfe_ctx *ctx, const uint8_t *target, int64_t tlen, const uint8_t *query,
                      int64_t qlen, const sfe_hsp *hsps, int64_t nhsps,
                      const sfe_ydrop_params *params, sfe_galign *out, int64_t cap,
                      int64_t *nout, sfe_ydrop_stats *stats);
/* Test hook (host only, needs no GPU; no counterpart in the paper): the
 * gapped stage's index of committed alignment boxes. Adds the n boxes in
 * order, then answers for each of the m queries, given as (strand, t, q)
 * triples, whether a box contains it (same strand, tstart <= t < tend and
 * qstart <= q < qend): inside[k] = 1 or 0. SFE_EINVAL on NULL arrays with
 * n or m above 0, or on a negative count. */
int sfe_test_committed_boxes(const sfe_galign *boxes, int64_t n, const int32_t *queries,
                             int64_t m, uint8_t *inside);

/*
 * Allocation-free variant of sfe_ungapped_xdrop (the paper has no counterpart:
 * this entry point exists for callers of the library, not for the method).
 *
 * For callers that cannot allocate device memory: code running inside
 * another framework's memory pool or under a hard memory budget, plugins whose
 * host owns every device allocation, and latency-critical paths where an
 * allocation and its implicit synchronisation are not allowed. The call never
 * allocates: no cudaMalloc, cudaFree, stream-ordered allocation or context.
 * Its scratch is one statically sized device array in the library (about
 * 13 MiB), which every GPU that loads the library holds until the process
 * exits.
 *
 * Limits: tlen and qlen at most 2^20 bases each, nhits at most 2^17; larger
 * inputs return SFE_ELIMIT before any GPU work.
 *
 * Arguments: target (tlen bases), query (qlen bases) and hits (nhits records,
 * any order) must be device pointers; bases are ASCII (input_codes = 0) or
 * codes 0..3 (input_codes = 1); seed_pattern NULL means 12of19 (only its span
 * is used). scores, X and hsp_thresh as in sfe_ungapped_xdrop. hsps: device
 * buffer of cap records, filled with the HSPs sorted by (strand, tpos, qpos,
 * len, score); if more than cap are found, *nhsps receives the needed count,
 * the buffer's contents are unspecified and SFE_EOVERFLOW is returned. stats
 * may be NULL. Work is queued on `stream` (a cudaStream_t; NULL is the legacy
 * default stream) and the call returns after it completes. The output equals
 * sfe_ungapped_xdrop's on the same inputs.
 *
 * The first call on a device looks up the array's device address for that
 * device (with that device current); make that first call before capturing
 * the stream into a graph. Every call shares the one array and the call clears
 * the parts that must start at zero, so calls whose GPU work overlaps (two host
 * threads, or two streams of one device) race on it and must be serialised by
 * the caller. Errors are reported through the return code only (this call sets
 * no message for sfe_last_error).
 */
int sfe_ungapped_xdrop_static(const uint8_t *target, int64_t tlen, const uint8_t *query,
                              int64_t qlen, const char *seed_pattern, int32_t input_codes,
                              const sfe_hit *hits, int64_t nhits, const int32_t scores[16],
                              int32_t X, int32_t hsp_thresh, sfe_hsp *hsps, int64_t cap,
                              int64_t *nhsps, sfe_stats *stats, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SFE_H */
