// The work predictor of the learned schedule: an MLP that reads a seed hit's
// sequence context and predicts the log of its extension length.
//
// Input: the 32 diagonal columns on each side of the seed (left flank
// t - 32 .. t - 1 against q - 32 .. q - 1, right flank t + span .. t + span + 31
// against the same offsets from q + span), each one-hot over its substitution
// class, the XOR of the two 2-bit codes (0 match, 2 transition, 1 and 3 the
// two kinds of transversion); a column that leaves either sequence is all
// zero. 64 columns x 4 = 256 inputs. Layers: 256 -> 64 (ReLU) -> 64 (ReLU) -> 1.
// Target: log(1 + bases the X-drop scored on both sides). The first layer is a
// gather: at most 64 inputs are one, so its output is the bias plus the sum of
// those rows of W1.
//
// Training keeps FP32 parameters and runs here: one warp per sample (lane j
// owns hidden units j and j + 32), a fused forward/backward kernel whose blocks
// accumulate weight gradients in shared memory before one atomic flush, and an
// Adam update. Inference uses FP16 weights with FP32 accumulation.
//
// Parameter layout (floats): W1[256][64], b1[64], W2[64][64], b2[64], W3[64], b3.
#include <cuda_fp16.h>

#include <cmath>

#include "sfe_internal.cuh"

namespace sfe {

namespace {

constexpr int IN = 256, H = 64;
constexpr int CTX = 32;  // columns per flank
constexpr int OFF_W1 = 0, OFF_B1 = IN * H, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H, NPARAM = OFF_B3 + 1;
constexpr int MLP_BLOCK = 256, MLP_WARPS = MLP_BLOCK / 32;

// Active one-hot inputs of a sample: lane l returns the input index of left
// column l (l * 4 + class) and of right column l ((32 + l) * 4 + class), or -1
// for a column outside the sequences.
__device__ __forceinline__ void context_inputs(const uint32_t *__restrict__ T, long long tlen,
                                               long long tb, const uint32_t *__restrict__ Q,
                                               long long qlen, long long qb, long long t,
                                               long long q, int span, int lane, int &in_l,
                                               int &in_r) {
    long long pt = t - CTX + lane, pq = q - CTX + lane;
    in_l = (pt >= 0 && pt < tlen && pq >= 0 && pq < qlen)
               ? lane * 4 + (int)(base_at(T, tb + pt) ^ base_at(Q, qb + pq))
               : -1;
    pt = t + span + lane;
    pq = q + span + lane;
    in_r = (pt >= 0 && pt < tlen && pq >= 0 && pq < qlen)
               ? (CTX + lane) * 4 + (int)(base_at(T, tb + pt) ^ base_at(Q, qb + pq))
               : -1;
}

struct SampleCtx {
    const uint32_t *T, *Q, *Qrc;
    long long tlen, qlen;
    const PairInfo *pairs;  // null: one pair (tlen, qlen above)
    int span;               // seed span
};

__device__ __forceinline__ void sample_inputs(const SampleCtx &sc, const sfe_ext_record &r,
                                              int lane, int &in_l, int &in_r) {
    long long tb = 0, qb = 0, tl = sc.tlen, ql = sc.qlen;
    if (sc.pairs) {
        const PairInfo P = sc.pairs[r.pair];
        tb = P.toff;
        qb = r.strand ? P.qoff_rc : P.qoff;
        tl = P.tlen;
        ql = P.qlen;
    }
    context_inputs(sc.T, tl, tb, r.strand ? sc.Qrc : sc.Q, ql, qb, r.t, r.q, sc.span, lane, in_l,
                   in_r);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Forward pass of one sample by one warp; returns the prediction and leaves
// the activations of units (lane, lane + 32) in z1/a1/z2/a2.
template <typename WT>
__device__ __forceinline__ float forward_warp(const WT *__restrict__ W1, const float *__restrict__ b1,
                                              const WT *__restrict__ W2, const float *__restrict__ b2,
                                              const WT *__restrict__ W3, float b3, int in_t,
                                              int in_q, int lane, float (&z1)[2], float (&a1)[2],
                                              float (&z2)[2], float (&a2)[2]) {
    z1[0] = b1[lane];
    z1[1] = b1[lane + 32];
    for (int k = 0; k < 32; k++) {
        const int it = __shfl_sync(0xffffffffu, in_t, k);
        const int iq = __shfl_sync(0xffffffffu, in_q, k);
        if (it >= 0) {
            z1[0] += (float)W1[it * H + lane];
            z1[1] += (float)W1[it * H + lane + 32];
        }
        if (iq >= 0) {
            z1[0] += (float)W1[iq * H + lane];
            z1[1] += (float)W1[iq * H + lane + 32];
        }
    }
    a1[0] = fmaxf(z1[0], 0.f);
    a1[1] = fmaxf(z1[1], 0.f);
    z2[0] = b2[lane];
    z2[1] = b2[lane + 32];
    for (int i = 0; i < H; i++) {
        const float ai = __shfl_sync(0xffffffffu, a1[i >> 5], i & 31);
        z2[0] += ai * (float)W2[i * H + lane];
        z2[1] += ai * (float)W2[i * H + lane + 32];
    }
    a2[0] = fmaxf(z2[0], 0.f);
    a2[1] = fmaxf(z2[1], 0.f);
    return warp_sum(a2[0] * (float)W3[lane] + a2[1] * (float)W3[lane + 32]) + b3;
}

__device__ __forceinline__ float target_of(const sfe_ext_record &r) {
    return logf(1.f + (float)(r.right + r.left));
}

// Loss (sum of squared errors) and, when grad != nullptr, the gradient of the
// mean squared error over n samples, accumulated per block in shared memory.
__global__ void __launch_bounds__(MLP_BLOCK) mlp_fwd_bwd(SampleCtx sc,
                                                         const sfe_ext_record *__restrict__ recs,
                                                         const uint32_t *__restrict__ perm,
                                                         long long n, const float *__restrict__ P,
                                                         float *__restrict__ grad,
                                                         float *__restrict__ preds,
                                                         double *__restrict__ loss) {
    extern __shared__ float gs[];  // NPARAM floats of block gradient (when grad)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (grad)
        for (int i = threadIdx.x; i < NPARAM; i += MLP_BLOCK) gs[i] = 0.f;
    __syncthreads();
    const float *W1 = P + OFF_W1, *b1 = P + OFF_B1, *W2 = P + OFF_W2, *b2 = P + OFF_B2,
                *W3 = P + OFF_W3;
    const float b3 = P[OFF_B3];
    const float inv_n = 1.f / (float)n;
    double lsum = 0.0;
    for (long long s = blockIdx.x * (long long)MLP_WARPS + w; s < n;
         s += (long long)gridDim.x * MLP_WARPS) {
        const sfe_ext_record r = recs[perm ? perm[s] : s];
        int in_t, in_q;
        sample_inputs(sc, r, lane, in_t, in_q);
        float z1[2], a1[2], z2[2], a2[2];
        const float y = forward_warp<float>(W1, b1, W2, b2, W3, b3, in_t, in_q, lane, z1, a1, z2,
                                            a2);
        const float err = y - target_of(r);
        if (lane == 0) {
            lsum += (double)err * err;
            if (preds) preds[s] = y;
        }
        if (!grad) continue;
        const float dy = 2.f * err * inv_n;
        // layer 3
        atomicAdd(&gs[OFF_W3 + lane], dy * a2[0]);
        atomicAdd(&gs[OFF_W3 + lane + 32], dy * a2[1]);
        if (lane == 0) atomicAdd(&gs[OFF_B3], dy);
        float dz2[2];
        dz2[0] = z2[0] > 0.f ? dy * W3[lane] : 0.f;
        dz2[1] = z2[1] > 0.f ? dy * W3[lane + 32] : 0.f;
        atomicAdd(&gs[OFF_B2 + lane], dz2[0]);
        atomicAdd(&gs[OFF_B2 + lane + 32], dz2[1]);
        // layer 2: dW2[i][j] += a1[i] dz2[j]; da1[i] = sum_j W2[i][j] dz2[j]
        float da1[2] = {0.f, 0.f};
        for (int i = 0; i < H; i++) {
            const float ai = __shfl_sync(0xffffffffu, a1[i >> 5], i & 31);
            if (ai != 0.f) {
                atomicAdd(&gs[OFF_W2 + i * H + lane], ai * dz2[0]);
                atomicAdd(&gs[OFF_W2 + i * H + lane + 32], ai * dz2[1]);
            }
            const float part = warp_sum(W2[i * H + lane] * dz2[0] + W2[i * H + lane + 32] * dz2[1]);
            if ((i & 31) == lane) da1[i >> 5] = part;
        }
        float dz1[2];
        dz1[0] = z1[0] > 0.f ? da1[0] : 0.f;
        dz1[1] = z1[1] > 0.f ? da1[1] : 0.f;
        atomicAdd(&gs[OFF_B1 + lane], dz1[0]);
        atomicAdd(&gs[OFF_B1 + lane + 32], dz1[1]);
        // layer 1: the rows of the active inputs
        for (int k = 0; k < 32; k++) {
            const int it = __shfl_sync(0xffffffffu, in_t, k);
            const int iq = __shfl_sync(0xffffffffu, in_q, k);
            if (it >= 0) {
                atomicAdd(&gs[OFF_W1 + it * H + lane], dz1[0]);
                atomicAdd(&gs[OFF_W1 + it * H + lane + 32], dz1[1]);
            }
            if (iq >= 0) {
                atomicAdd(&gs[OFF_W1 + iq * H + lane], dz1[0]);
                atomicAdd(&gs[OFF_W1 + iq * H + lane + 32], dz1[1]);
            }
        }
    }
    if (lane == 0 && lsum != 0.0) atomicAdd(loss, lsum);
    __syncthreads();
    if (grad)
        for (int i = threadIdx.x; i < NPARAM; i += MLP_BLOCK)
            if (gs[i] != 0.f) atomicAdd(&grad[i], gs[i]);
}

// Adam (Kingma and Ba 2015) with bias correction.
__global__ void adam_kernel(float *__restrict__ P, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// He-style initialisation from a counter-based hash (uniform, scaled by fan-in).
__global__ void init_kernel(float *__restrict__ P, unsigned long long seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float u = (float)(z >> 40) * (1.f / 16777216.f) * 2.f - 1.f;  // [-1, 1)
    float scale = 0.f;
    if (i < OFF_B1) scale = sqrtf(6.f / 64.f);        // 64 active inputs
    else if (i >= OFF_W2 && i < OFF_B2) scale = sqrtf(6.f / H);
    else if (i >= OFF_W3 && i < OFF_B3) scale = sqrtf(3.f / H);
    P[i] = (i == OFF_B3) ? 3.0f : u * scale;  // b3: a typical log length
}

// FP16 weights, FP32 biases: the inference model.
__global__ void pack_kernel16(const float *__restrict__ P, __half *__restrict__ w16,
                              float *__restrict__ b32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const bool is_bias = (i >= OFF_B1 && i < OFF_W2) || (i >= OFF_B2 && i < OFF_W3) || i == OFF_B3;
    if (is_bias)
        b32[i] = P[i];
    else
        w16[i] = __float2half_rn(P[i]);
}

// ---------------------------------------------------------------------------
// Inference on the tensor cores (mma.sync m16n8k16, FP16 inputs, FP32
// accumulation). One warp evaluates 16 samples: layer 1 is the dense product
// of the 16 x 256 one-hot inputs with W1 (16 k-steps x 8 n-tiles), layer 2
// the product of the 16 x 64 hidden activations, rounded to FP16, with W2 (4 x
// 8); the accumulator fragments of layer 1 are, register for register, the
// input fragments of layer 2. Weights sit in shared memory transposed (one row
// per hidden unit) with 8 halves of padding, so the eight rows a fragment load
// touches fall in different banks.
constexpr int MMA_WARPS = 4, MMA_BLOCK = MMA_WARPS * 32;
constexpr int W1T_LD = IN + 8, W2T_LD = H + 8;

struct MmaSmem {
    __half w1t[H * W1T_LD];
    __half w2t[H * W2T_LD];
    float b1[H], b2[H], w3[H];
    float b3;
    unsigned long long cls[MMA_WARPS][16][2];  // per sample, per flank: 32 classes (2 bits)
    uint32_t valid[MMA_WARPS][16][2];          // per sample, per flank: columns inside
};

__device__ void mma_load_weights(MmaSmem &sm, const __half *__restrict__ w16,
                                 const float *__restrict__ b32) {
    for (int i = threadIdx.x; i < IN * H; i += blockDim.x)  // W1[k][n] -> w1t[n][k]
        sm.w1t[(i % H) * W1T_LD + i / H] = w16[OFF_W1 + i];
    for (int i = threadIdx.x; i < H * H; i += blockDim.x)
        sm.w2t[(i % H) * W2T_LD + i / H] = w16[OFF_W2 + i];
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        sm.b1[i] = b32[OFF_B1 + i];
        sm.b2[i] = b32[OFF_B2 + i];
        sm.w3[i] = __half2float(w16[OFF_W3 + i]);
    }
    if (threadIdx.x == 0) sm.b3 = b32[OFF_B3];
}

// Classes (T xor Q) of the 32 columns of one flank of a hit, and which of
// them lie inside both sequences. side 0: t - 32 .. t - 1, side 1: t + span ..
__device__ __forceinline__ void flank(const uint32_t *__restrict__ T, long long tb, long long tl,
                                      const uint32_t *__restrict__ Qs, long long qb,
                                      long long ql, long long t, long long q, int span, int side,
                                      unsigned long long &cls, uint32_t &valid) {
    const long long pt = side ? t + span : t - 32, pq = side ? q + span : q - 32;
    cls = 0;
    valid = 0;
    // reads stay inside the padded buffers only for flanks that start within
    // 32 bases before a sequence and not after its end
    if (pt < -32 || pt > tl || pq < -32 || pq > ql) return;
    const unsigned long long tw =
        (unsigned long long)win16(T, tb + pt) | ((unsigned long long)win16(T, tb + pt + 16) << 32);
    const unsigned long long qw = (unsigned long long)win16(Qs, qb + pq) |
                                  ((unsigned long long)win16(Qs, qb + pq + 16) << 32);
    cls = tw ^ qw;
    const long long lo = max(0LL, max(-pt, -pq));          // first column inside
    const long long hi = min(32LL, min(tl - pt, ql - pq));  // one past the last
    if (hi > lo) valid = (hi >= 32 ? 0xFFFFFFFFu : ((1u << hi) - 1u)) & (0xFFFFFFFFu << lo);
}

__device__ __forceinline__ uint32_t onehot2(const MmaSmem &sm, int w, int row, int col, int slot) {
    const int side = col >> 5, i = col & 31;
    const uint32_t c = (uint32_t)(sm.cls[w][row][side] >> (2 * i)) & 3u;
    const bool v = (sm.valid[w][row][side] >> i) & 1u;
    return ((v && c == (uint32_t)slot) ? 0x3C00u : 0u) |  // FP16 1.0 in the low half
           ((v && c == (uint32_t)slot + 1u) ? 0x3C000000u : 0u);
}

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// The network on the 16 samples whose flanks are in sm.cls[w] / sm.valid[w].
// Lane l returns the predictions of samples l / 4 and l / 4 + 8 (every lane
// of a quad holds the same two).
__device__ __forceinline__ void mma_forward16(const MmaSmem &sm, int w, int lane, float &y_lo,
                                              float &y_hi) {
    const int g = lane >> 2, tq = lane & 3;
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll 2
    for (int kk = 0; kk < IN / 16; kk++) {
        const int col0 = kk * 4 + (tq >> 1), slot = (tq & 1) * 2;
        const uint32_t a0 = onehot2(sm, w, g, col0, slot), a1 = onehot2(sm, w, g + 8, col0, slot);
        const uint32_t a2 = onehot2(sm, w, g, col0 + 2, slot);
        const uint32_t a3 = onehot2(sm, w, g + 8, col0 + 2, slot);
        const int k0 = kk * 16 + tq * 2;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const __half *row = sm.w1t + (j * 8 + g) * W1T_LD + k0;
            mma16816(acc[j], a0, a1, a2, a3, *reinterpret_cast<const uint32_t *>(row),
                     *reinterpret_cast<const uint32_t *>(row + 8));
        }
    }
    // bias, ReLU, FP16: the A fragments of layer 2
    uint32_t h[8][2];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const int c = j * 8 + tq * 2;
        h[j][0] = pack_half2(fmaxf(acc[j][0] + sm.b1[c], 0.f), fmaxf(acc[j][1] + sm.b1[c + 1], 0.f));
        h[j][1] = pack_half2(fmaxf(acc[j][2] + sm.b1[c], 0.f), fmaxf(acc[j][3] + sm.b1[c + 1], 0.f));
    }
    float acc2[8][4];
#pragma unroll
    for (int j = 0; j < 8; j++) acc2[j][0] = acc2[j][1] = acc2[j][2] = acc2[j][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < H / 16; kk++) {
        const int k0 = kk * 16 + tq * 2;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const __half *row = sm.w2t + (j * 8 + g) * W2T_LD + k0;
            mma16816(acc2[j], h[2 * kk][0], h[2 * kk][1], h[2 * kk + 1][0], h[2 * kk + 1][1],
                     *reinterpret_cast<const uint32_t *>(row),
                     *reinterpret_cast<const uint32_t *>(row + 8));
        }
    }
    float plo = 0.f, phi = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const int c = j * 8 + tq * 2;
        plo += fmaxf(acc2[j][0] + sm.b2[c], 0.f) * sm.w3[c] +
               fmaxf(acc2[j][1] + sm.b2[c + 1], 0.f) * sm.w3[c + 1];
        phi += fmaxf(acc2[j][2] + sm.b2[c], 0.f) * sm.w3[c] +
               fmaxf(acc2[j][3] + sm.b2[c + 1], 0.f) * sm.w3[c + 1];
    }
    plo += __shfl_xor_sync(0xffffffffu, plo, 1);
    plo += __shfl_xor_sync(0xffffffffu, plo, 2);
    phi += __shfl_xor_sync(0xffffffffu, phi, 1);
    phi += __shfl_xor_sync(0xffffffffu, phi, 2);
    y_lo = plo + sm.b3;
    y_hi = phi + sm.b3;
}

// A hit's record fields from its walk word.
__device__ __forceinline__ sfe_ext_record hit_record(uint64_t h, const WalkParams &wp) {
    const uint32_t word = (uint32_t)(h >> 32);
    sfe_ext_record r;
    long long D, qlen;
    if (wp.pairs) {
        r.pair = (int)(word >> (wp.dbits + 1));
        r.strand = (int)((word >> wp.dbits) & 1u);
        D = (long long)(word & ((1u << wp.dbits) - 1u));
        qlen = wp.pairs[r.pair].qlen;
    } else {
        r.pair = 0;
        r.strand = wp.strand;
        D = (long long)(word & 0x7FFFFFFFu);
        qlen = wp.qlen;
    }
    r.t = (int)(uint32_t)h;
    r.q = (int)((long long)(uint32_t)h - D + qlen - wp.span);
    r.right = r.left = 0;
    return r;
}

// Flanks of a record into the warp's sample slot s (lane: s + 16 * side).
__device__ __forceinline__ void record_flank(MmaSmem &sm, int w, int s, int side,
                                             const SampleCtx &sc, const sfe_ext_record &r) {
    long long tb = 0, qb = 0, tl = sc.tlen, ql = sc.qlen;
    if (sc.pairs) {
        const PairInfo P = sc.pairs[r.pair];
        tb = P.toff;
        qb = r.strand ? P.qoff_rc : P.qoff;
        tl = P.tlen;
        ql = P.qlen;
    }
    flank(sc.T, tb, tl, r.strand ? sc.Qrc : sc.Q, qb, ql, r.t, r.q, sc.span, side,
          sm.cls[w][s][side], sm.valid[w][s][side]);
}

// Predictions of the FP16 model for extension records, 16 per warp.
__global__ void __launch_bounds__(MMA_BLOCK) mlp_predict_mma(SampleCtx sc,
                                                             const sfe_ext_record *__restrict__ recs,
                                                             long long n,
                                                             const __half *__restrict__ w16,
                                                             const float *__restrict__ b32,
                                                             float *__restrict__ preds) {
    __shared__ MmaSmem sm;
    mma_load_weights(sm, w16, b32);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long groups = (n + 15) / 16;
    for (long long grp = blockIdx.x * (long long)MMA_WARPS + w; grp < groups;
         grp += (long long)gridDim.x * MMA_WARPS) {
        const long long idx = grp * 16 + (lane & 15);
        const int side = lane >> 4;
        if (idx < n) {
            record_flank(sm, w, lane & 15, side, sc, recs[idx]);
        } else {
            sm.cls[w][lane & 15][side] = 0;
            sm.valid[w][lane & 15][side] = 0;
        }
        __syncwarp();
        float ylo, yhi;
        mma_forward16(sm, w, lane, ylo, yhi);
        if ((lane & 3) == 0) {
            const long long r0 = grp * 16 + (lane >> 2), r1 = r0 + 8;
            if (r0 < n) preds[r0] = ylo;
            if (r1 < n) preds[r1] = yhi;
        }
        __syncwarp();
    }
}

// Predicted work of each chunk of hits for the learned schedule: exp of the
// prediction for the chunk's first hit times the chunk's hit count, 16 chunks
// per warp. Key: (~work, chunk), so an ascending sort puts the most work
// first; chunks past a device-side hit count get the largest key.
__global__ void __launch_bounds__(MMA_BLOCK) chunk_predict_mma(
    const uint64_t *__restrict__ hits, uint32_t n, uint32_t chunk, uint32_t nchunks,
    WalkParams wp, const __half *__restrict__ w16, const float *__restrict__ b32,
    uint64_t *__restrict__ keys) {
    __shared__ MmaSmem sm;
    mma_load_weights(sm, w16, b32);
    __syncthreads();
    if (wp.nd) n = (uint32_t)min((unsigned long long)n, *wp.nd);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // one pair: wp.Q is already the walked strand's query
    const SampleCtx sc{wp.T, wp.Q, wp.pairs ? wp.Qrc : wp.Q, wp.tlen, wp.qlen, wp.pairs, wp.span};
    const long long groups = ((long long)nchunks + 15) / 16;
    for (long long grp = blockIdx.x * (long long)MMA_WARPS + w; grp < groups;
         grp += (long long)gridDim.x * MMA_WARPS) {
        const long long k = grp * 16 + (lane & 15);
        const int side = lane >> 4;
        const unsigned long long i0 = (unsigned long long)k * chunk;
        if (k < nchunks && i0 < n) {
            record_flank(sm, w, lane & 15, side, sc, hit_record(hits[i0], wp));
        } else {
            sm.cls[w][lane & 15][side] = 0;
            sm.valid[w][lane & 15][side] = 0;
        }
        __syncwarp();
        float ylo, yhi;
        mma_forward16(sm, w, lane, ylo, yhi);
        if ((lane & 3) == 0) {
#pragma unroll
            for (int hsel = 0; hsel < 2; hsel++) {
                const long long kc = grp * 16 + (lane >> 2) + 8 * hsel;
                if (kc >= nchunks) continue;
                const unsigned long long c0 = (unsigned long long)kc * chunk;
                if (c0 >= n) {
                    keys[kc] = (0xFFFFFFFFull << 32) | (uint32_t)kc;
                    continue;
                }
                const float len = (float)min((unsigned long long)chunk, n - c0);
                const float work = expf(fminf(hsel ? yhi : ylo, 20.f)) * len;
                const uint32_t qk = (uint32_t)fmaxf(1.f, fminf(work * 16.f, 4.0e9f));
                keys[kc] = ((uint64_t)(0xFFFFFFFFu - qk) << 32) | (uint32_t)kc;
            }
        }
        __syncwarp();
    }
}

// A record is usable when its pair and strand exist; positions need no
// check (context reads outside a sequence are zero inputs).
__global__ void validate_records(const sfe_ext_record *__restrict__ recs, long long n, int npairs,
                                 uint32_t *status) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const sfe_ext_record r = recs[i];
    if (r.pair < 0 || r.pair >= npairs || (r.strand != 0 && r.strand != 1))
        atomicOr(status, ST_BAD_HIT);
}

// Sort keys of a random permutation: (hash(seed, epoch, i), i).
__global__ void perm_keys(long long n, unsigned long long seed, int epoch,
                          uint64_t *__restrict__ keys) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long z = seed ^ (0xD1B54A32D192ED03ull * (unsigned long long)(epoch + 1));
    z += 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    keys[i] = (z & 0xFFFFFFFF00000000ull) | (uint64_t)(uint32_t)i;
}

__global__ void perm_extract(const uint64_t *__restrict__ keys, long long n,
                             uint32_t *__restrict__ perm) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) perm[i] = (uint32_t)keys[i];
}

unsigned blocks_for(long long threads, int block) {
    return (unsigned)((threads + block - 1) / block);
}

}  // namespace

// Inference grids: four CTAs per SM at most (the kernels stride over sample
// groups).
static long long predict_grid(long long want) {
    return max(1LL, min(want, 4LL * device_sms()));
}

cudaError_t launch_mlp_predict16(const uint32_t *T, long long tlen, const uint32_t *Q,
                                 const uint32_t *Qrc, long long qlen, const PairInfo *pairs,
                                 int span, const sfe_ext_record *recs, long long n,
                                 const void *model, float *preds, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const SampleCtx sc{T, Q, Qrc, tlen, qlen, pairs, span};
    const __half *w16 = reinterpret_cast<const __half *>(model);
    const float *b32 = reinterpret_cast<const float *>(reinterpret_cast<const char *>(model) +
                                                       ((size_t)NPARAM * 2 + 255) / 256 * 256);
    const long long groups = (n + 15) / 16;
    const long long want = (groups + MMA_WARPS - 1) / MMA_WARPS;
    g_launches++;
    mlp_predict_mma<<<(unsigned)predict_grid(want), MMA_BLOCK, 0, st>>>(sc, recs, n, w16, b32,
                                                                       preds);
    return cudaGetLastError();
}

cudaError_t launch_validate_records(const sfe_ext_record *recs, long long n, int npairs,
                                    uint32_t *status, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    g_launches++;
    validate_records<<<blocks_for(n, 256), 256, 0, st>>>(recs, n, npairs, status);
    return cudaGetLastError();
}

cudaError_t launch_perm(long long n, unsigned long long seed, int epoch, uint64_t *ka,
                        uint64_t *kb, void *tmp, uint32_t *perm, uint32_t *status,
                        cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    g_launches++;
    perm_keys<<<blocks_for(n, 256), 256, 0, st>>>(n, seed, epoch, ka);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bool in_b = false;
    e = radix_sort(ka, kb, nullptr, nullptr, n, 32, 64, tmp, &in_b, status, st);
    if (e != cudaSuccess) return e;
    g_launches++;
    perm_extract<<<blocks_for(n, 256), 256, 0, st>>>(in_b ? kb : ka, n, perm);
    return cudaGetLastError();
}

cudaError_t launch_chunk_predict(const uint64_t *hits, long long n, uint32_t chunk,
                                 uint32_t nchunks, const WalkParams &wp, const void *model,
                                 uint64_t *keys, cudaStream_t st) {
    const __half *w16 = reinterpret_cast<const __half *>(model);
    const float *b32 = reinterpret_cast<const float *>(reinterpret_cast<const char *>(model) +
                                                       ((size_t)NPARAM * 2 + 255) / 256 * 256);
    const long long groups = ((long long)nchunks + 15) / 16;
    const long long want = (groups + MMA_WARPS - 1) / MMA_WARPS;
    g_launches++;
    chunk_predict_mma<<<(unsigned)predict_grid(want), MMA_BLOCK, 0, st>>>(
        hits, (uint32_t)n, chunk, nchunks, wp, w16, b32, keys);
    return cudaGetLastError();
}

// Inference model blob: NPARAM halves, then NPARAM floats (biases used).
size_t mlp_model_bytes() { return ((size_t)NPARAM * 2 + 255) / 256 * 256 + (size_t)NPARAM * 4; }
int mlp_param_count() { return NPARAM; }

cudaError_t launch_mlp_init(float *P, unsigned long long seed, cudaStream_t st) {
    g_launches++;
    init_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(P, seed);
    return cudaGetLastError();
}

cudaError_t launch_mlp_pack(const float *P, void *model, cudaStream_t st) {
    __half *w16 = reinterpret_cast<__half *>(model);
    float *b32 = reinterpret_cast<float *>(reinterpret_cast<char *>(model) +
                                           ((size_t)NPARAM * 2 + 255) / 256 * 256);
    g_launches++;
    pack_kernel16<<<(NPARAM + 255) / 256, 256, 0, st>>>(P, w16, b32);
    return cudaGetLastError();
}

cudaError_t launch_mlp_fwd_bwd(const uint32_t *T, long long tlen, const uint32_t *Q,
                               const uint32_t *Qrc, long long qlen, const PairInfo *pairs,
                               int span, const sfe_ext_record *recs, const uint32_t *perm,
                               long long n, const float *P, float *grad, float *preds,
                               double *loss, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const SampleCtx sc{T, Q, Qrc, tlen, qlen, pairs, span};
    const size_t smem = grad ? (size_t)NPARAM * 4 : 0;
    static std::atomic<unsigned long long> attr;
    cudaError_t ae = once_per_device(attr, [] {
        return cudaFuncSetAttribute(mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    NPARAM * 4);
    });
    if (ae != cudaSuccess) return ae;
    const int sms = device_sms();
    // about 4 samples per warp: each block flushes its whole gradient once
    long long want = (n + 4 * MLP_WARPS - 1) / (4 * MLP_WARPS);
    long long grid = want < 2LL * sms ? want : 2LL * sms;
    if (grid < 1) grid = 1;
    g_launches++;
    mlp_fwd_bwd<<<(unsigned)grid, MLP_BLOCK, smem, st>>>(sc, recs, perm, n, P, grad, preds, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *P, const float *g, float *m, float *v, float lr, int step,
                        cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    g_launches++;
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(P, g, m, v, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

}  // namespace sfe
