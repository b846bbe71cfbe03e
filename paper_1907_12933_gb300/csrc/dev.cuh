// dev.cuh -- device-side views shared by the kernels of the verifier.
//
// Layout in HBM (one net, one result workspace per query):
//   net:    W_l fp32 [H_l][H_{l-1}] (row = neuron, Eq. 1), W_l^T fp32, b_l,
//           per-row norms, bf16/fp16/e4m3 copies for the tensor screens
//   query:  ub/hb (FP64 potentials/outputs of the unperturbed image, all
//           layers back to back), per-neuron screen constants (fp32),
//           layer-1 delta tables tab[p][d][j] (fp32), counters, masks,
//           verdict bitmap, tie list
//   queues: (query, point) pairs waiting for a tighter pass
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace vbmc {

constexpr int kMaxL = 8;
constexpr int kMaxS = 16;
constexpr int kMaxR = 255;
constexpr int kMaxWidth = 1024;
constexpr double kTau = 1e-9;  // tie band of margins and potentials

enum { ACT_IDENTITY = 0, ACT_SIGMOID = 1, ACT_RELU = 2 };

// Device error codes latched in Counters::err.
enum : unsigned {
    DERR_PIXELS = 1u,    // pixel list not distinct / out of range
    DERR_QUEUE = 2u,     // a recheck queue overflowed
    DERR_TIES = 4u,      // tie list truncated (not an error for results)
    DERR_TC_WAIT = 8u,   // a tensor-core pipeline wait gave up
};

struct NetView {
    int L;                  // weight layers
    int act;                // hidden activation
    int total;              // non-input neurons
    int hmax;               // max width over layers 1..L
    int dims[kMaxL + 1];    // H_0..H_L
    int noff[kMaxL + 2];    // neuron offset of layer l (1..L) in concatenated vectors
    long long ssoff[kMaxL + 1];  // SS bit offset of pair (l, l+1), l = 1..L-1
    int flip_words, ss_words;
    const float* W[kMaxL + 1];   // W[l], l = 1..L: [H_l][H_{l-1}]
    const float* WT[kMaxL + 1];  // [H_{l-1}][H_l]
    const float* b[kMaxL + 1];
    const float* rownorm[kMaxL + 1];  // ||W_l,i||_2 (rounded up)
    float lamfrob[kMaxL + 1];         // lambda * ||W_l||_F (rounded up; lambda: Lipschitz
                                      // constant of the hidden activation)
    float gam[kMaxL + 1];             // gamma_{H_{l-1}} = n u / (1 - n u), u = 2^-24
    float lamsig[kMaxL + 1];          // lambda * sigma_max(W_l) (rounded up)
    float sig[kMaxL + 1];             // sigma_max(W_l) (rounded up)
    float frob[kMaxL + 1];            // ||W_l||_F (rounded up)
    const float* pairw;               // [H_L][H_L]: ||W_L,D - W_L,o||_2 (rounded up)
    // launch shapes (0: the built-in choice; set by vbmc_autotune)
    int simt_var_range, simt_var_gather;    // FP32 pass variant, 1..6
    int simt_ctas_range, simt_ctas_gather;  // FP32 pass CTAs per SM
    int df_ctas;                            // double-float pass CTAs per SM
};

struct Counters {
    unsigned long long n_adv;
    unsigned long long first;    // smallest adversarial index
    unsigned long long n_ties;
    unsigned long long n_q[4];   // entries pushed to queue level 0 (tensor split), 1 (FP32),
                                 // 2 (double-float), 3 (FP64)
    unsigned long long n_points;
    unsigned int err;
    int D;
    double base_margin;
    unsigned long long t0;          // %globaltimer at the start of the query's prologue
    unsigned long long t_final;     // ... when its result became final (0: not yet)
    unsigned long long work;        // unfinished units: screen tiles not yet done plus
                                    // queued points not yet resolved (see work_done)
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

enum { FILTER_L2 = 1, FILTER_SHELL = 2 };
enum { PROP_ARGMAX = 0, PROP_THRESHOLD = 1 };

struct QueryView {
    int s, k, R, qid;
    int filter;             // FILTER_L2 | FILTER_SHELL, 0: every point of the box
    long long l2max;        // FILTER_L2: largest sum over the pixels of dv^2 (grey levels^2)
    int prop;               // PROP_ARGMAX (Eq. 10) or PROP_THRESHOLD (Eq. 11)
    double V;               // PROP_THRESHOLD: the reference value V
    unsigned long long n_points, lo, hi;  // space size and checked range
    unsigned long long ntiles;            // screen tiles of this query (time-to-verdict)
    unsigned long long budget_ns;         // time budget of the call from the query's prologue
                                          // (0: none); see claim_tile
    const uint8_t* image;   // H_0 grey levels (device)
    const int* pix_in;      // s pixel indices as given (device)
    int* pix;               // validated copy
    int* dv;                // [s][R]: clamp(v_p + d - k, 0, 255) - v_p
    double* ub;             // [total] FP64 potentials of the unperturbed image
    double* hb;             // [total] FP64 outputs (act(ub); output layer: ub)
    double* eub;            // [total] bound on |ub - exact| from the FP64 base pass
    float* ub32;            // [total] fp32(ub)
    float* dub;             // [total] value error of fl(ub) (+ layer-1 table-sum error)
    float* thr;             // [total] sign-certainty threshold: dub + 2 tau, or +inf when
                            //         |ub| < tau (every evaluation is a sign tie)
    float* c1;              // [total] delta-activation constants (see screen_simt.cu)
    float* c2;
    float* tab;             // [s][R][H_1] layer-1 deltas W_1[j][p] * dv / 255
    float* kvec;            // [kMaxL+1] per-layer constant error-norm terms
    uint32_t* cpos;         // [kMaxL+1][32] tensor screen: columns whose sign never changes
    uint32_t* cneg;         //   (pos: output change = input change; neg: output stays 0)
    // Compacted columns of the tensor screen (one query per call): the neurons of
    // hidden layer l that are not of the class "neg" come first, in order, so
    // the dense layers run over them only (a "neg" neuron's change is 0 at every
    // point of the box, so dropping it changes no product).
    int compact;            // 1: the set-up of this call built the compacted operands below
                            //    (the tensor screen, and the FP32 pass of the same call, read them)
    int* perm;              // [total]: layer l at noff[l]: compacted position -> neuron
    int* kc;                // [kMaxL+1]: layer l's compacted width, a multiple of 64
    float* tabc;            // [s][R][H_1]: tab in compacted column order
    float* w1c;             // [kMaxS][H_1]: W_1[perm_1[j']][pix_p], compacted order
    float* wtc[kMaxL + 1];  // l >= 2: W_l^T [H_{l-1}][H_l], rows and columns compacted
                            // (the output layer keeps its columns)
    // Column constants of the tensor screen per hidden neuron, two float4 each:
    // (fl(ub), ||Wq_i||, ||W_i - Wq_i||, ||W_i - Wq_i - Wlo_i||) and (thr, c1, c2,
    // class), with the delta-ReLU constants of the class folded in (pos: 0, -inf;
    // neg: -inf, 0) and class 0 pos, 1 neg, 2 cross. kcol in neuron order,
    // kcolc in compacted order (padding positions "neg").
    float4* kcol;           // [total][2]
    float4* kcolc;          // [total][2]
    Counters* cnt;
    uint32_t* bitmap;       // verdict bits (nullptr: off)
    unsigned long long bitmap_bits;
    uint32_t *flip, *flip_tie, *ss, *ss_tie;  // nullptr: coverage off
    unsigned long long* ties;
    unsigned int ties_cap;
};

struct QEntry {
    unsigned long long t;
    unsigned int q;
    unsigned int pad;
};

struct Queue {
    QEntry* e;
    unsigned long long* count;  // entries pushed (may exceed cap: overflow)
    unsigned long long cap;
};

__device__ __forceinline__ void set_bit_atomic(uint32_t* w, unsigned long long b) {
    atomicOr(&w[b >> 5], 1u << (unsigned)(b & 31));
}

// Time to verdict. Counters::work starts at the query's number of screen
// tiles; every queued point adds one (in the push helpers below) and every
// finished tile or resolved queued point takes one away, after the pushes it
// caused. The update that takes it to zero stamps t_final: from then on no
// pass changes the query's result. The push helpers fence after their
// increments, and callers reach work_done only after a barrier that follows
// their pushes, so the count cannot reach zero while a push is outstanding.
__device__ __forceinline__ void work_done(Counters* c, unsigned long long n) {
    __threadfence();
    if (n && atomicAdd(&c->work, 0ull - n) == n) c->t_final = globaltimer_ns();
}

__device__ __forceinline__ void queue_push(const Queue& Q, unsigned long long t, unsigned q,
                                           Counters* cnt, int level) {
    unsigned long long i = atomicAdd(Q.count, 1ull);
    atomicAdd(&cnt->n_q[level], 1ull);
    atomicAdd(&cnt->work, 1ull);
    __threadfence();
    if (i < Q.cap) {
        QEntry e;
        e.t = t;
        e.q = q;
        e.pad = 0;
        Q.e[i] = e;
    } else {
        atomicOr(&cnt->err, DERR_QUEUE);
    }
}

// Warp-cooperative push: every lane of the warp calls it (converged); lanes with
// want == true get one slot each from a single atomic per warp. Lanes may hold
// points of different queries: each query's counters get its own lanes' count.
__device__ __forceinline__ void queue_push_warp(const Queue& Q, bool want, unsigned long long t,
                                                unsigned q, Counters* cnt, int level) {
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(Q.count, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (want) {
        const unsigned peers = __match_any_sync(m, reinterpret_cast<unsigned long long>(cnt));
        if (lane == __ffs(peers) - 1) {
            atomicAdd(&cnt->n_q[level], (unsigned long long)__popc(peers));
            atomicAdd(&cnt->work, (unsigned long long)__popc(peers));
            __threadfence();
        }
    }
    if (want) {
        const unsigned long long i = base + __popc(m & ((1u << lane) - 1u));
        if (i < Q.cap) {
            QEntry e;
            e.t = t;
            e.q = q;
            e.pad = 0;
            Q.e[i] = e;
        } else {
            atomicOr(&cnt->err, DERR_QUEUE);
        }
    }
}

// Set a bit that many points set: read first, write only if still clear.
__device__ __forceinline__ void set_bit_once(uint32_t* w, unsigned long long b) {
    const uint32_t m = 1u << (unsigned)(b & 31);
    if (!(*reinterpret_cast<volatile uint32_t*>(&w[b >> 5]) & m)) atomicOr(&w[b >> 5], m);
}

// Record a certainly adversarial (non-tie) point.
__device__ __forceinline__ void record_adversarial(const QueryView& Q, unsigned long long t) {
    atomicAdd(&Q.cnt->n_adv, 1ull);
    atomicMin(&Q.cnt->first, t);
    if (Q.bitmap && t < Q.bitmap_bits) set_bit_atomic(Q.bitmap, t);
}

// Tile claims of the persistent first passes. With a claim counter the tiles
// are handed out in increasing order, one atomicAdd each, so the tiles a launch
// has taken always form a prefix [0, min(counter, ntiles)) of its tile list;
// a claim checks the time budget (deadline in %globaltimer ns, 0: none)
// before it takes a tile, so none is taken past the deadline and every tile
// taken is finished. Without a counter the tiles are statically strided.
constexpr unsigned long long kNoTile = ~0ull;

__device__ __forceinline__ unsigned long long claim_tile(unsigned long long* ctr, unsigned long long i,
                                                         unsigned long long ntiles, unsigned long long deadline) {
    if (!ctr) {
        const unsigned long long g = (unsigned long long)blockIdx.x + i * (unsigned long long)gridDim.x;
        return g < ntiles ? g : kNoTile;
    }
    if (deadline && globaltimer_ns() > deadline) return kNoTile;
    const unsigned long long g = atomicAdd(ctr, 1ull);
    return g < ntiles ? g : kNoTile;
}

// Mixed-radix decode: first pixel most significant.
__device__ __forceinline__ void decode_digits(unsigned long long t, int s, int R, int* d) {
    if (t < 0xFFFFFFFFull) {
        unsigned tt = (unsigned)t;
        for (int p = s - 1; p >= 0; --p) {
            d[p] = (int)(tt % (unsigned)R);
            tt /= (unsigned)R;
        }
    } else {
        for (int p = s - 1; p >= 0; --p) {
            d[p] = (int)(t % (unsigned long long)R);
            t /= (unsigned long long)R;
        }
    }
}

// Eq. 11 in a screen: the point is misclassified iff y_D < V and y_o > V for
// some other output o. thr_side gives the side of V that output value y lies on
// for certain: +1 above, -1 below, 0 undecided, where e bounds |y - exact| plus
// the 2 tau tie slack; the 2^-22 (|y| + |V|) term covers the FP32 roundings of
// V, of y and of y - V.
__device__ __forceinline__ int thr_side(float y, float V, float e) {
    const float t = __fmaf_ru(0x1p-22f, __fadd_ru(fabsf(y), fabsf(V)), e);
    return y - V > t ? 1 : (V - y > t ? -1 : 0);
}

// Verdict from the sides: 0 certainly not misclassified (y_D above V, or every
// other output below V), 1 certainly misclassified (y_D below V and some other
// output above V), 2 undecided (a tighter pass decides).
__device__ __forceinline__ int thr_verdict(bool d_above, bool d_below, bool other_above, bool others_below) {
    if (d_above || others_below) return 0;
    return d_below && other_above ? 1 : 2;
}

// The point's digits pass the query's filter: the perturbed image within the
// Euclidean ball sum_p dv_p^2 <= l2max (Eq. 9 on the grid, clipped steps), and
// on the box's boundary max_p |d_p - k| = k (one shell of the k-shell order).
__device__ __forceinline__ bool in_filter(const QueryView& Q, const int* d) {
    if (!Q.filter) return true;
    if (Q.filter & FILTER_L2) {
        long long s2 = 0;
        for (int p = 0; p < Q.s; ++p) {
            const long long v = Q.dv[p * Q.R + d[p]];
            s2 += v * v;
        }
        if (s2 > Q.l2max) return false;
    }
    if (Q.filter & FILTER_SHELL) {
        bool on = Q.k == 0;
        for (int p = 0; p < Q.s; ++p) on = on || d[p] == 0 || d[p] == Q.R - 1;
        if (!on) return false;
    }
    return true;
}

}  // namespace vbmc
