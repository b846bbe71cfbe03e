// api.cu -- host runtime behind include/vbmc.h.
//
// A vbmc_net holds the weights on the device plus the per-row norms that the
// screens' error bounds use. A vbmc_result is a reusable workspace: the
// per-query constants, the counters, the coverage masks, the verdict bitmap,
// the tie list and the recheck queues, all allocated once. A verify call
// enqueues: prologue (FP64 base pass, tables, constants) -> screen pass over
// every point -> tighter passes over the queued points -> FP64 pass.
#include "../../include/vbmc.h"
#include "dev.cuh"
#include "launch.h"
#include "tc.h"
#include "wide.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace vbmc;

namespace {

thread_local std::string g_err;

vbmc_status fail(vbmc_status st, const std::string& msg) {
    g_err = msg;
    return st;
}

#define VB_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? VBMC_ERR_OOM : VBMC_ERR_CUDA, \
                        std::string(#call ": ") + cudaGetErrorString(e_));              \
    } while (0)

float round_up_f(double x) {
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, INFINITY);
    return f;
}

uint64_t space_size(int s, int k) {
    const uint64_t R = (uint64_t)(2 * k + 1);
    uint64_t n = 1;
    for (int p = 0; p < s; ++p) {
        if (n > (1ull << 62) / R) return 0;
        n *= R;
    }
    return n;
}

template <class T>
cudaError_t dalloc(T** p, size_t n, std::vector<void*>& owned) {
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e == cudaSuccess) owned.push_back((void*)*p);
    return e;
}

}  // namespace

struct vbmc_net {
    NetView v{};
    std::vector<void*> owned;
    int n_sm = 0;
    int device = 0;
    TcNet tc{};  // tensor-core copies (built on first use per precision)
    WideNet wide{};  // rounded copies for the wide-layer path (built on first use per type)
    std::vector<std::vector<float>> hW, hb;  // host copies for tensor-core set-up
};

// Shared state of results created together by vbmc_result_create_batch: the
// query views and counters of all members back to back (so one launch can
// cover every query), one staging buffer for the queries' images and pixel
// lists, and the recheck queues the batch passes share.
struct BatchArena {
    int nq = 0;
    int refs = 0;
    QueryView* d_qs = nullptr;      // member views by slot (what the result handles read)
    QueryView* d_qs_run = nullptr;  // the same views in the batch call's schedule order
    Counters* d_cnt = nullptr;
    Counters* h_cnt = nullptr;  // pinned
    unsigned long long* d_tp = nullptr;
    uint8_t* d_stage = nullptr;
    size_t stage_stride = 0;
    unsigned long long* d_qcount = nullptr;
    unsigned long long* d_claim = nullptr;  // tile claims of each wave's first pass
    QEntry* d_queue[4] = {nullptr, nullptr, nullptr, nullptr};
    uint64_t queue_cap = 0;
    cudaEvent_t ev[7] = {};  // start, prologue, screen, end, split, FP32, double-float
    cudaEvent_t evw = nullptr;       // marks between waves (not read)
    cudaStream_t gstream = nullptr;  // graph capture needs a capturable (non-legacy) stream
    cudaEvent_t gev = nullptr;
    // the pass chain of the last graph call, instantiated, and the shapes it was
    // captured for (kernel arguments depend only on them; the queries' data and
    // tile prefixes are copied in before each launch)
    cudaGraphExec_t gexec = nullptr;
    std::string gsig;
    std::vector<void*> owned;
};

struct vbmc_result {
    BatchArena* arena = nullptr;
    int slot = 0;
    const vbmc_net* net = nullptr;
    vbmc_caps caps{};
    std::vector<void*> owned;
    QueryView hq{};           // host copy of the device view
    QueryView* d_q = nullptr;
    Counters* d_cnt = nullptr;
    Counters* h_cnt = nullptr;  // pinned
    uint8_t* d_image = nullptr;
    int* d_pix_in = nullptr;
    unsigned long long* d_tp = nullptr;  // tile prefix {0, n_tiles}
    unsigned long long* d_qcount = nullptr;  // 4 queue counters
    QEntry* d_queue[4] = {nullptr, nullptr, nullptr, nullptr};
    double* d_margin = nullptr;
    WideWork ww{};  // chunk workspace of the wide-layer path (caps.wide_chunk; allocated at creation)
    unsigned long long* d_tiles = nullptr;  // VBMC_MAX_TILES counters of vbmc_tile_counts
    TcQueryWork tw{};  // compacted operands of the fused tensor screen (single-query calls)
    bool have_tw = false;
    unsigned long long* d_claim = nullptr;  // tile claim counter of the first pass
    unsigned long long* h_claim = nullptr;  // pinned copy after the call
    unsigned long long ntiles = 0;          // first-pass tiles of the last call
    int tile_pts = 0;                       // points per first-pass tile (0: no claim counter)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_pro = nullptr, ev_scr = nullptr;
    cudaEvent_t ev_split = nullptr, ev_f32 = nullptr, ev_df = nullptr;  // after each recheck pass
    cudaStream_t last_stream = nullptr;
    bool pending = false;
    bool have_result = false;
    int flip_words = 0, ss_words = 0;
    // query of the last call (host copy)
    std::vector<uint8_t> image;
    std::vector<int32_t> pixels;
    int s = 0, k = 0;
    uint64_t lo = 0, hi = 0, n_space = 0;
    vbmc_options opt{};
    vbmc_summary sum{};
    vbmc_status last_status = VBMC_OK;
};

extern "C" const char* vbmc_last_error(void) { return g_err.c_str(); }

namespace vbmc {
const NetView* net_view(const vbmc_net* net) { return &net->v; }
vbmc_status set_error(vbmc_status st, const char* msg) { return fail(st, msg); }
}  // namespace vbmc

extern "C" vbmc_status vbmc_net_create(const vbmc_mlp_desc* desc, vbmc_net** out) {
    if (!desc || !out) return fail(VBMC_ERR_ARG, "null argument");
    *out = nullptr;
    const int L = desc->n_layers;
    if (L < 1 || L > kMaxL) return fail(VBMC_ERR_ARG, "n_layers must be in [1, 8]");
    if (!desc->dims || !desc->W || !desc->b) return fail(VBMC_ERR_ARG, "null dims/W/b");
    if (desc->hidden_act < 0 || desc->hidden_act > 2) return fail(VBMC_ERR_ARG, "bad activation");
    for (int l = 0; l <= L; ++l)
        if (desc->dims[l] < 1 || (l > 0 && desc->dims[l] > kMaxWidth) || desc->dims[l] > (1 << 24))
            return fail(VBMC_ERR_ARG, "layer width out of range");
    if (desc->dims[L] < 2) return fail(VBMC_ERR_ARG, "output layer needs at least 2 classes");
    for (int l = 0; l < L; ++l)
        if (!desc->W[l] || !desc->b[l]) return fail(VBMC_ERR_ARG, "null weight pointer");

    vbmc_net* n = new vbmc_net();
    NetView& v = n->v;
    v.L = L;
    v.act = desc->hidden_act;
    for (int l = 0; l <= L; ++l) v.dims[l] = desc->dims[l];
    v.total = 0;
    v.hmax = 0;
    for (int l = 1; l <= L; ++l) {
        v.noff[l] = v.total;
        v.total += v.dims[l];
        v.hmax = std::max(v.hmax, v.dims[l]);
    }
    v.noff[L + 1] = v.total;
    long long ss = 0;
    for (int l = 1; l < L; ++l) {
        v.ssoff[l] = ss;
        ss += (long long)v.dims[l] * v.dims[l + 1];
    }
    v.flip_words = (v.total + 31) / 32;
    v.ss_words = (int)std::max<long long>(1, (ss + 31) / 32);
    const double lam = desc->hidden_act == VBMC_ACT_SIGMOID ? 0.25 : 1.0;
    cudaGetDevice(&n->device);
    cudaDeviceGetAttribute(&n->n_sm, cudaDevAttrMultiProcessorCount, n->device);
    n->hW.resize(L + 1);
    n->hb.resize(L + 1);
    for (int l = 1; l <= L; ++l) {
        const int K = v.dims[l - 1], N = v.dims[l];
        const float* W = desc->W[l - 1];
        const float* b = desc->b[l - 1];
        n->hW[l].assign(W, W + (size_t)N * K);
        n->hb[l].assign(b, b + N);
        std::vector<float> WT((size_t)N * K), rn(N);
        double frob2 = 0.0;
        for (int i = 0; i < N; ++i) {
            double r2 = 0.0;
            for (int j = 0; j < K; ++j) {
                const double w = W[(size_t)i * K + j];
                if (!std::isfinite(w)) {
                    vbmc_net_free(n);
                    return fail(VBMC_ERR_ARG, "non-finite weight");
                }
                r2 += w * w;
                WT[(size_t)j * N + i] = W[(size_t)i * K + j];
            }
            rn[i] = round_up_f(std::sqrt(r2) * (1.0 + 1e-12));
            frob2 += r2;
        }
        v.lamfrob[l] = round_up_f(lam * std::sqrt(frob2) * (1.0 + 1e-12));
        v.frob[l] = round_up_f(std::sqrt(frob2) * (1.0 + 1e-12));
        if (l >= 2) {
            std::vector<double> Wd((size_t)N * K);
            for (size_t e = 0; e < Wd.size(); ++e) Wd[e] = W[e];
            const double sg = spectral_bound(Wd, N, K);
            if (!(sg > 0.0) && frob2 > 0.0) {
                vbmc_net_free(n);
                return fail(VBMC_ERR_CUDA, "spectral-norm bound failed");
            }
            v.sig[l] = round_up_f(sg);
            v.lamsig[l] = round_up_f(lam * sg);
        }
        if (l == L) {
            std::vector<float> pw((size_t)N * N);
            for (int D = 0; D < N; ++D)
                for (int o = 0; o < N; ++o) {
                    double d2 = 0.0;
                    for (int j = 0; j < K; ++j) {
                        const double d = (double)W[(size_t)D * K + j] - (double)W[(size_t)o * K + j];
                        d2 += d * d;
                    }
                    pw[(size_t)D * N + o] = round_up_f(std::sqrt(d2) * (1.0 + 1e-12));
                }
            float* dpw = nullptr;
            if (dalloc(&dpw, pw.size(), n->owned) != cudaSuccess ||
                cudaMemcpy(dpw, pw.data(), sizeof(float) * pw.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
                vbmc_net_free(n);
                return fail(VBMC_ERR_OOM, "net_create: pair norms");
            }
            v.pairw = dpw;
        }
        const double u = std::ldexp(1.0, -24);
        v.gam[l] = round_up_f(K * u / (1.0 - K * u));
        float *dW, *dWT, *db, *drn;
        cudaError_t e = dalloc(&dW, (size_t)N * K, n->owned);
        if (e == cudaSuccess) e = dalloc(&dWT, (size_t)N * K, n->owned);
        if (e == cudaSuccess) e = dalloc(&db, N, n->owned);
        if (e == cudaSuccess) e = dalloc(&drn, N, n->owned);
        if (e == cudaSuccess) e = cudaMemcpy(dW, W, sizeof(float) * N * K, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dWT, WT.data(), sizeof(float) * N * K, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(db, b, sizeof(float) * N, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(drn, rn.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            vbmc_net_free(n);
            return fail(VBMC_ERR_OOM, std::string("net_create: ") + cudaGetErrorString(e));
        }
        v.W[l] = dW;
        v.WT[l] = dWT;
        v.b[l] = db;
        v.rownorm[l] = drn;
    }
    // tensor-core operands and bound constants, so that verify calls allocate nothing
    for (int prec : {VBMC_PREC_BF16, VBMC_PREC_FP16}) {
        if (!tc_supported(v, prec)) continue;
        vbmc_status st = tc_build(n->tc, v, n->hW, n->hb, prec);
        if (st != VBMC_OK) {
            vbmc_net_free(n);
            return fail(st, "tensor-core set-up failed");
        }
    }
    *out = n;
    return VBMC_OK;
}

extern "C" vbmc_status vbmc_net_free(vbmc_net* net) {
    if (!net) return VBMC_OK;
    tc_free(net->tc);
    wide_free(net->wide);
    for (void* p : net->owned) cudaFree(p);
    delete net;
    return VBMC_OK;
}

extern "C" vbmc_status vbmc_mask_words(const vbmc_net* net, size_t* fw, size_t* sw) {
    if (!net) return fail(VBMC_ERR_ARG, "null net");
    if (fw) *fw = (size_t)net->v.flip_words;
    if (sw) *sw = (size_t)net->v.ss_words;
    return VBMC_OK;
}

namespace {

vbmc_status create_result(const vbmc_net* net, const vbmc_caps* caps, BatchArena* arena, int slot,
                          vbmc_result** out) {
    if (!net || !caps || !out) return fail(VBMC_ERR_ARG, "null argument");
    *out = nullptr;
    if (caps->max_s < 0 || caps->max_s > kMaxS) return fail(VBMC_ERR_ARG, "max_s out of range");
    if (caps->max_k < 0 || caps->max_k > VBMC_MAX_K) return fail(VBMC_ERR_ARG, "max_k out of range");
    vbmc_result* r = new vbmc_result();
    r->net = net;
    r->caps = *caps;
    r->arena = arena;
    r->slot = slot;
    if (arena) arena->refs++;  // released by vbmc_result_free, also on the failure path
    const NetView& v = net->v;
    const int S = std::max(1, caps->max_s), RM = 2 * caps->max_k + 1;
    const size_t T = v.total;
    r->flip_words = v.flip_words;
    r->ss_words = v.ss_words;
    QueryView& q = r->hq;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t n) {
        if (e == cudaSuccess) e = dalloc(p, n, r->owned);
    };
    if (arena) {
        r->d_q = arena->d_qs + slot;
        r->d_cnt = arena->d_cnt + slot;
    } else {
        A(&r->d_q, 1);
        A(&r->d_cnt, 1);
    }
    A(&r->d_image, (size_t)v.dims[0]);
    A(&r->d_pix_in, (size_t)S);
    A(&q.pix, (size_t)S);
    A(&q.dv, (size_t)S * RM);
    A(&q.ub, T);
    A(&q.hb, T);
    A(&q.eub, T);
    A(&q.ub32, T);
    A(&q.dub, T);
    A(&q.thr, T);
    A(&q.c1, T);
    A(&q.c2, T);
    A(&q.tab, (size_t)S * RM * v.dims[1]);
    A(&q.kvec, (size_t)kMaxL + 1);
    A(&q.cpos, (size_t)(kMaxL + 1) * 32);
    A(&q.cneg, (size_t)(kMaxL + 1) * 32);
    A(&q.flip, (size_t)v.flip_words);
    A(&q.flip_tie, (size_t)v.flip_words);
    A(&q.ss, (size_t)v.ss_words);
    A(&q.ss_tie, (size_t)v.ss_words);
    A(&q.ties, (size_t)std::max<uint32_t>(1, caps->ties_cap));
    A(&r->d_tp, 2);
    A(&r->d_qcount, 4);
    A(&r->d_margin, 1);
    if (caps->max_points) A(&q.bitmap, (size_t)((caps->max_points + 31) / 32));
    // members of a batch keep small queues of their own (the batch shares the arena's)
    uint64_t qc = std::max<uint64_t>(1, caps->queue_cap);
    if (arena) qc = std::min<uint64_t>(qc, 1u << 16);
    r->caps.queue_cap = qc;
    for (int i = 0; i < 4; ++i) A(&r->d_queue[i], (size_t)qc);
    A(&r->d_tiles, (size_t)VBMC_MAX_TILES);
    A(&r->d_claim, 1);
    // compacted columns of the fused tensor screen (calls with one query)
    const bool tcnet = tc_supported(v, VBMC_PREC_BF16) || tc_supported(v, VBMC_PREC_FP16);
    const bool fused = !arena && tcnet;
    if (tcnet) A(&q.kcol, 2 * T);
    if (fused) {
        A(&q.kcolc, 2 * T);
        A(&q.perm, T);
        A(&q.kc, (size_t)2 * (kMaxL + 1));
        A(&q.tabc, (size_t)S * RM * v.dims[1]);
        A(&q.w1c, (size_t)kMaxS * v.dims[1]);
        for (int l = 2; l <= v.L; ++l) A(&q.wtc[l], (size_t)v.dims[l - 1] * v.dims[l]);
    }
    if (e == cudaSuccess) e = cudaMallocHost((void**)&r->h_cnt, sizeof(Counters));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&r->h_claim, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreate(&r->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&r->ev1);
    if (e == cudaSuccess) e = cudaEventCreate(&r->ev_pro);
    if (e == cudaSuccess) e = cudaEventCreate(&r->ev_scr);
    if (e == cudaSuccess) e = cudaEventCreate(&r->ev_split);
    if (e == cudaSuccess) e = cudaEventCreate(&r->ev_f32);
    if (e == cudaSuccess) e = cudaEventCreate(&r->ev_df);
    if (e != cudaSuccess) {
        vbmc_result_free(r);
        return fail(VBMC_ERR_OOM, std::string("result_create: ") + cudaGetErrorString(e));
    }
    if (fused) {
        const vbmc_status ts = tc_query_work_alloc(r->tw, v);
        if (ts != VBMC_OK) {
            vbmc_result_free(r);
            return fail(ts, "result_create: compacted tensor-screen weights");
        }
        r->have_tw = true;
    }
    // the wide-layer tensor path's chunk workspace: sized here so that verify
    // calls allocate nothing (batch members: only when asked for explicitly)
    if (wide_supported(v) && caps->wide_chunk >= 0 && !(arena && caps->wide_chunk == 0)) {
        unsigned long long chunk = (unsigned long long)caps->wide_chunk;
        if (chunk == 0) {
            const uint64_t box = space_size(caps->max_s, caps->max_k);
            chunk = (box == 0 || box > (1ull << 20)) ? (1ull << 20) : box;
        }
        const vbmc_status ws = wide_work_alloc(r->ww, v, chunk);
        if (ws != VBMC_OK) {
            vbmc_result_free(r);
            return fail(ws, "result_create: wide-layer workspace (lower caps.wide_chunk, or -1 for none)");
        }
    }
    q.cnt = r->d_cnt;
    q.bitmap_bits = caps->max_points;
    q.ties_cap = caps->ties_cap;
    *out = r;
    return VBMC_OK;
}

void arena_release(BatchArena* a) {
    if (!a || --a->refs > 0) return;
    for (void* p : a->owned) cudaFree(p);
    if (a->h_cnt) cudaFreeHost(a->h_cnt);
    for (cudaEvent_t ev : a->ev)
        if (ev) cudaEventDestroy(ev);
    if (a->evw) cudaEventDestroy(a->evw);
    if (a->gev) cudaEventDestroy(a->gev);
    if (a->gexec) cudaGraphExecDestroy(a->gexec);
    if (a->gstream) cudaStreamDestroy(a->gstream);
    delete a;
}

}  // namespace

extern "C" vbmc_status vbmc_result_create(const vbmc_net* net, const vbmc_caps* caps,
                                          vbmc_result** out) {
    return create_result(net, caps, nullptr, 0, out);
}

extern "C" vbmc_status vbmc_result_create_batch(const vbmc_net* net, const vbmc_caps* caps,
                                                int32_t nq, vbmc_result** out) {
    if (!net || !caps || !out || nq <= 0) return fail(VBMC_ERR_ARG, "null argument or nq <= 0");
    BatchArena* ar = new BatchArena();
    ar->nq = nq;
    ar->refs = 1;  // held by this call until every member exists
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t n) {
        if (e == cudaSuccess) e = dalloc(p, n, ar->owned);
    };
    ar->stage_stride = ((size_t)net->v.dims[0] + sizeof(int32_t) * kMaxS + 15) & ~size_t(15);
    A(&ar->d_qs, (size_t)nq);
    A(&ar->d_qs_run, (size_t)nq);
    A(&ar->d_cnt, (size_t)nq);
    A(&ar->d_tp, 2 * (size_t)nq + 2);  // one tile prefix per wave, back to back
    A(&ar->d_stage, ar->stage_stride * (size_t)nq);
    A(&ar->d_qcount, 4);
    A(&ar->d_claim, 1);
    ar->queue_cap = std::max<uint64_t>(1, caps->queue_cap);
    for (int i = 0; i < 4; ++i) A(&ar->d_queue[i], (size_t)ar->queue_cap);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ar->h_cnt, sizeof(Counters) * (size_t)nq);
    for (int i = 0; i < 7 && e == cudaSuccess; ++i) e = cudaEventCreate(&ar->ev[i]);
    if (e == cudaSuccess) e = cudaEventCreate(&ar->evw);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ar->gstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ar->gev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        arena_release(ar);
        return fail(VBMC_ERR_OOM, std::string("result_create_batch: ") + cudaGetErrorString(e));
    }
    for (int i = 0; i < nq; ++i) {
        vbmc_status st = create_result(net, caps, ar, i, &out[i]);
        if (st != VBMC_OK) {
            for (int j = 0; j < i; ++j) vbmc_result_free(out[j]);
            arena_release(ar);
            return st;
        }
    }
    arena_release(ar);  // the members hold it now
    return VBMC_OK;
}

extern "C" vbmc_status vbmc_result_free(vbmc_result* r) {
    if (!r) return VBMC_OK;
    if (r->pending && r->last_stream) cudaStreamSynchronize(r->last_stream);
    for (void* p : r->owned) cudaFree(p);
    wide_work_free(r->ww);
    tc_query_work_free(r->tw);
    arena_release(r->arena);
    if (r->h_cnt) cudaFreeHost(r->h_cnt);
    if (r->h_claim) cudaFreeHost(r->h_claim);
    if (r->ev0) cudaEventDestroy(r->ev0);
    if (r->ev1) cudaEventDestroy(r->ev1);
    if (r->ev_pro) cudaEventDestroy(r->ev_pro);
    if (r->ev_scr) cudaEventDestroy(r->ev_scr);
    for (cudaEvent_t x : {r->ev_split, r->ev_f32, r->ev_df})
        if (x) cudaEventDestroy(x);
    delete r;
    return VBMC_OK;
}

namespace {

vbmc_status check_query_shape(const vbmc_result* r, int s, int k, uint64_t lo, uint64_t hi,
                              const vbmc_options* opt, uint64_t* n_out, uint64_t* hi_out) {
    if (s < 0 || s > r->caps.max_s) return fail(VBMC_ERR_ARG, "s exceeds the result's max_s");
    if (k < 0 || k > r->caps.max_k) return fail(VBMC_ERR_ARG, "k exceeds the result's max_k");
    const uint64_t n = space_size(s, k);
    if (n == 0) return fail(VBMC_ERR_ARG, "R^s does not fit below 2^62");
    if (hi == 0) hi = n;
    if (hi > n || lo > hi) return fail(VBMC_ERR_ARG, "range [lo, hi) outside [0, R^s)");
    if (opt && opt->bitmap && hi > r->caps.max_points)
        return fail(VBMC_ERR_ARG, "verdict bitmap larger than the result's max_points");
    if (opt && (opt->precision < 0 || opt->precision > VBMC_PREC_FP8))
        return fail(VBMC_ERR_ARG, "bad precision");
    *n_out = n;
    *hi_out = hi;
    return VBMC_OK;
}

// Tiles of the first pass for each query (sets QueryView::ntiles) and their
// prefix; 0 tiles for the FP64 path (one block per point there).
std::vector<unsigned long long> tile_prefix(const NetView& v, int precision, QueryView* hq, int nq) {
    const int MT = precision == VBMC_PREC_FP64 ? 0
                   : precision == VBMC_PREC_FP32 ? (nq == 1 && small_supported(v) ? small_tile_points()
                                                                                 : simt_tile_points(v))
                                                 : tc_tile_points();
    std::vector<unsigned long long> tp((size_t)nq + 1, 0);
    for (int i = 0; i < nq; ++i) {
        const unsigned long long base = hq[i].lo & ~31ull;
        unsigned long long t = (MT && hq[i].hi > hq[i].lo) ? (hq[i].hi - base + MT - 1) / MT : 0;
        if (precision == VBMC_PREC_FP8 || ((precision == VBMC_PREC_BF16 || precision == VBMC_PREC_FP16) &&
                                           !tc_supported(v, precision)))
            t = hq[i].hi > hq[i].lo ? 1 : 0;  // the wide-layer path: one unit, its chunk loop
        hq[i].ntiles = t;
        tp[i + 1] = tp[i] + t;
    }
    return tp;
}

// Stages of enqueue_passes: per-query set-up (prologue and tensor-core column
// classes) and the passes over the points of [lo, hi).
enum { STAGE_SETUP = 1, STAGE_PASSES = 2, STAGE_ALL = 3 };

// Every pass for nq queries whose views (and tile prefix) are already on the
// device. ev: start, after the prologue, after the first pass, end, after the
// split tensor pass, after the FP32 pass, after the double-float pass. The set-up
// stage resets the counters and clears the masks and the verdict bitmap over
// [0, hi); everything else it computes depends on the box, not on [lo, hi),
// so one set-up over the whole space serves passes over any sub-ranges.
vbmc_status enqueue_passes(vbmc_net* net, QueryView* d_qs, const QueryView* hq, int nq,
                           const unsigned long long* d_tp, unsigned long long ntiles,
                           unsigned long long* d_qcount, QEntry* const* d_queue,
                           unsigned long long cap, const cudaEvent_t* ev, const vbmc_options& opt,
                           cudaStream_t st, bool capturing = false, int stages = STAGE_ALL,
                           WideWork* ww = nullptr, TcQueryWork* tw = nullptr,
                           unsigned long long* d_claim = nullptr) {
    if (nq != 1) tw = nullptr;  // compacted columns are per query: single-query calls only
    const NetView& v = net->v;
    // inside a stream capture an event record must be an explicit graph node
    const unsigned evflag = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    auto record = [&](cudaEvent_t e) { return cudaEventRecordWithFlags(e, st, evflag); };
    int max_sr = 0;
    bool any = false;
    for (int i = 0; i < nq; ++i) {
        max_sr = std::max(max_sr, hq[i].s * hq[i].R);
        any = any || hq[i].hi > hq[i].lo;
    }
    // 16-bit screens: the fused kernel where it fits, else the wide-layer path;
    // E4M3 always takes the wide-layer path
    const bool tensor16 = opt.precision == VBMC_PREC_BF16 || opt.precision == VBMC_PREC_FP16;
    const bool wide = opt.precision == VBMC_PREC_FP8 || (tensor16 && !tc_supported(v, opt.precision));
    const bool tensor = tensor16 && !wide;
    const int wtype = wide_type(opt.precision);
    if (wide && any) {
        if (nq != 1 || !ww) return fail(VBMC_ERR_UNSUPPORTED, "the wide-layer tensor screen serves one query per call");
        if (!wide_supported(v))
            return fail(VBMC_ERR_UNSUPPORTED,
                        "tensor-core screen does not support this net/precision (wide layers: ReLU, hidden widths "
                        "a multiple of 256 up to 1024, at most 32 outputs)");
        vbmc_status fs = wide_build(net->wide, v, net->hW, wtype);
        if (fs != VBMC_OK) return fail(fs, "wide-layer tensor set-up failed (self-test or weight preparation)");
        if (!ww->chunk)
            return fail(VBMC_ERR_STATE, "the result has no wide-layer workspace (created with caps.wide_chunk = -1, "
                                        "or as a batch member without one)");
    }
    VB_CUDA(cudaMemsetAsync(d_qcount, 0, sizeof(unsigned long long) * 4, st));
    VB_CUDA(record(ev[0]));
    if (stages & STAGE_SETUP) launch_prologue(v, d_qs, nq, max_sr, st);
    VB_CUDA(record(ev[1]));
    if (tensor && any) {
        if (!tc_supported(v, opt.precision))
            return fail(VBMC_ERR_UNSUPPORTED, "tensor-core screen does not support this net/precision");
        vbmc_status sst = tc_build(net->tc, v, net->hW, net->hb, opt.precision);
        if (sst != VBMC_OK) return fail(sst, "tensor-core set-up failed");
        if (stages & STAGE_SETUP) tc_launch_query_setup(net->tc, v, d_qs, nq, opt.precision, st, tw);
    }
    if (!(stages & STAGE_PASSES)) return VBMC_OK;
    // queue levels: 0 tensor split pass, 1 FP32 pass, 2 double-float pass, 3 FP64 pass
    Queue qsplit{d_queue[0], d_qcount + 0, cap};
    Queue q32{d_queue[1], d_qcount + 1, cap};
    Queue qdf{d_queue[2], d_qcount + 2, cap};
    Queue q64{d_queue[3], d_qcount + 3, cap};
    auto record_rest = [&]() -> cudaError_t {  // passes that did not run take no time
        for (int i : {4, 5, 6}) {
            const cudaError_t e = record(ev[i]);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    if (any && wide) {
        // the chunk loop interleaves the screen and the rechecks: all of it counts as screen
        vbmc_status fs = wide_run(net->wide, wtype, *ww, v, d_qs, hq[0].lo, hq[0].hi, d_qcount, d_queue, cap,
                                  net->n_sm, st);
        if (fs != VBMC_OK) return fail(fs, "wide-layer tensor screen launch failed");
        VB_CUDA(record(ev[2]));
        VB_CUDA(record_rest());
    } else if (any && opt.precision == VBMC_PREC_FP64) {
        for (int i = 0; i < nq; ++i)
            if (hq[i].hi > hq[i].lo)
                launch_fp64(v, d_qs + i, 1, nullptr, nullptr, 0, hq[i].lo, hq[i].hi, net->n_sm, st);
        VB_CUDA(record(ev[2]));
        VB_CUDA(record_rest());
    } else if (any) {
        if (opt.precision == VBMC_PREC_FP32) {
            if (simt_tile_points(v) == 0) return fail(VBMC_ERR_UNSUPPORTED, "layer width above 1024");
            launch_screen_simt(v, d_qs, nq, d_tp, ntiles, nullptr, nullptr, 0, qdf, 2, net->n_sm, st,
                               (nq == 1 && small_supported(v)) ? nullptr : d_claim);
            VB_CUDA(record(ev[2]));
            VB_CUDA(record(ev[4]));
            VB_CUDA(record(ev[5]));
        } else {
            // one query: screen -> split tensor pass -> FP32; many: screen -> FP32 directly
            vbmc_status sst = tc_launch_screen(net->tc, v, d_qs, nq, d_tp, ntiles, opt.precision,
                                   nq == 1 ? qsplit : q32, nq == 1 ? 0 : 1, net->n_sm, st, tw, d_claim);
            if (sst != VBMC_OK)
                return fail(sst, std::string("tensor-core screen launch failed: ") + cudaGetErrorString(cudaGetLastError()));
            VB_CUDA(record(ev[2]));
            if (nq == 1) {
                sst = tc_launch_gather(net->tc, v, d_qs, d_queue[0], d_qcount + 0, cap, opt.precision,
                                       q32, net->n_sm, st, tw);
                if (sst != VBMC_OK)
                    return fail(sst, std::string("tensor-core split pass launch failed: ") +
                                         cudaGetErrorString(cudaGetLastError()));
            }
            VB_CUDA(record(ev[4]));
            launch_screen_simt(v, d_qs, nq, nullptr, 0, d_queue[1], d_qcount + 1, cap, qdf, 2,
                               net->n_sm, st);
            VB_CUDA(record(ev[5]));
        }
        launch_df(v, d_qs, nq, d_queue[2], d_qcount + 2, cap, q64, 3, net->n_sm, st);
        VB_CUDA(record(ev[6]));
        launch_fp64(v, d_qs, nq, d_queue[3], d_qcount + 3, cap, 0, 0, net->n_sm, st);
    } else {
        VB_CUDA(record(ev[2]));
        VB_CUDA(record_rest());
    }
    launch_stamp_final(d_qs, nq, st);
    VB_CUDA(cudaGetLastError());
    VB_CUDA(record(ev[3]));
    return VBMC_OK;
}

// Point filter and property of a query (the fields of vbmc_query beyond the box).
struct QueryExtra {
    int filter = 0;
    long long l2max = 0;
    int prop = PROP_ARGMAX;
    double V = 0.0;
};

vbmc_status query_extra(const vbmc_query& q, QueryExtra* x) {
    if ((q.filter & ~(VBMC_FILTER_L2 | VBMC_FILTER_SHELL)) || ((q.filter & VBMC_FILTER_L2) && q.l2_max < 0))
        return fail(VBMC_ERR_ARG, "bad filter (VBMC_FILTER_L2 needs l2_max >= 0)");
    if (q.property != VBMC_PROP_ARGMAX && q.property != VBMC_PROP_THRESHOLD)
        return fail(VBMC_ERR_ARG, "bad property");
    if (q.property == VBMC_PROP_THRESHOLD && !std::isfinite(q.threshold))
        return fail(VBMC_ERR_ARG, "threshold must be finite");
    x->filter = q.filter;
    x->l2max = (long long)q.l2_max;
    x->prop = q.property == VBMC_PROP_THRESHOLD ? PROP_THRESHOLD : PROP_ARGMAX;
    x->V = x->prop == PROP_THRESHOLD ? q.threshold : 0.0;
    return VBMC_OK;
}

QueryView make_view(const vbmc_result* r, const uint8_t* d_image, const int* d_pix, int s, int k,
                    uint64_t lo, uint64_t hi, uint64_t n, const vbmc_options& opt, int qid,
                    const QueryExtra& x = QueryExtra()) {
    QueryView q = r->hq;
    q.filter = x.filter;
    q.l2max = x.l2max;
    q.prop = x.prop;
    q.V = x.V;
    q.s = s;
    q.k = k;
    q.R = 2 * k + 1;
    q.qid = qid;
    q.n_points = n;
    q.lo = lo;
    q.hi = hi;
    q.image = d_image;
    q.pix_in = d_pix;
    if (!opt.coverage) q.flip = q.flip_tie = q.ss = q.ss_tie = nullptr;
    if (!opt.bitmap) q.bitmap = nullptr;
    return q;
}

// Enqueue the full pipeline for one query whose image/pixels are on the device.
vbmc_status enqueue(vbmc_net* net, vbmc_result* r, const uint8_t* d_image, const int* d_pix, int s,
                    int k, uint64_t lo, uint64_t hi, uint64_t n, const vbmc_options& opt,
                    cudaStream_t st, const QueryExtra& x = QueryExtra()) {
    QueryView q = make_view(r, d_image, d_pix, s, k, lo, hi, n, opt, 0, x);
    q.budget_ns = opt.time_budget_ms > 0.0 ? (unsigned long long)(opt.time_budget_ms * 1e6) : 0ull;
    std::vector<unsigned long long> tp = tile_prefix(net->v, opt.precision, &q, 1);
    // the first pass takes its tiles from the claim counter on the fused tensor
    // screen and the FP32 path (not on small nets): the checked prefix follows
    const bool tensor16 = opt.precision == VBMC_PREC_BF16 || opt.precision == VBMC_PREC_FP16;
    const bool claims = (tensor16 && tc_supported(net->v, opt.precision)) ||
                        (opt.precision == VBMC_PREC_FP32 && !small_supported(net->v));
    r->ntiles = tp[1];
    r->tile_pts = claims ? (tensor16 ? tc_tile_points() : simt_tile_points(net->v)) : 0;
    VB_CUDA(cudaMemcpyAsync(r->d_q, &q, sizeof(QueryView), cudaMemcpyHostToDevice, st));
    VB_CUDA(cudaMemcpyAsync(r->d_tp, tp.data(), sizeof(unsigned long long) * 2, cudaMemcpyHostToDevice, st));
    const cudaEvent_t ev[7] = {r->ev0, r->ev_pro, r->ev_scr, r->ev1, r->ev_split, r->ev_f32, r->ev_df};
    vbmc_status sst = enqueue_passes(net, r->d_q, &q, 1, r->d_tp, tp[1], r->d_qcount, r->d_queue,
                                     std::max<uint64_t>(1, r->caps.queue_cap), ev, opt, st, false, STAGE_ALL,
                                     &r->ww, r->have_tw ? &r->tw : nullptr, claims ? r->d_claim : nullptr);
    if (sst != VBMC_OK) return sst;
    VB_CUDA(cudaMemcpyAsync(r->h_cnt, r->d_cnt, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    if (claims)
        VB_CUDA(cudaMemcpyAsync(r->h_claim, r->d_claim, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    r->last_stream = st;
    r->pending = true;
    r->have_result = true;
    r->s = s;
    r->k = k;
    r->lo = lo;
    r->hi = hi;
    r->n_space = n;
    r->opt = opt;
    return VBMC_OK;
}

void fill_summary(vbmc_result* r, const Counters& c, float ms, float ms_p, float ms_s,
                  const float* ms_pass = nullptr) {
    vbmc_summary& s = r->sum;
    std::memset(&s, 0, sizeof(s));
    s.D = c.D;
    s.base_margin = c.base_margin;
    s.n_points = c.n_points;  // points of [lo, hi) that pass the query's filter
    s.n_adversarial = c.n_adv;
    s.first_witness = c.first;
    s.n_ties = c.n_ties;
    for (int i = 0; i < 4; ++i) s.n_recheck[i] = c.n_q[i];
    s.ms_device = ms;
    s.ms_prologue = ms_p;
    s.ms_screen = ms_s;
    s.ms_recheck = ms - ms_p - ms_s;
    for (int i = 0; i < 4; ++i) s.ms_pass[i] = ms_pass ? ms_pass[i] : 0.0;
    s.ms_to_verdict = c.t_final > c.t0 ? (double)(c.t_final - c.t0) * 1e-6 : 0.0;
    // the checked prefix: tiles [0, claims) of the first pass (all of them unless
    // the time budget stopped the claims)
    s.checked_hi = r->hi;
    if (r->tile_pts > 0 && *r->h_claim < r->ntiles) {
        const uint64_t end = (r->lo & ~31ull) + *r->h_claim * (uint64_t)r->tile_pts;
        s.checked_hi = std::max<uint64_t>(r->lo, std::min<uint64_t>(r->hi, end));
        if (!(r->opt.time_budget_ms > 0.0)) s.checked_hi = r->hi;  // no budget: every tile was taken
        else if (s.n_points == r->hi - r->lo) s.n_points = s.checked_hi - r->lo;  // no filter: count the prefix
    }
    if (r->lo != 0 || s.checked_hi != r->n_space) s.verdict = VBMC_PARTIAL;
    else if (c.n_adv) s.verdict = VBMC_UNSAFE;
    else if (c.n_ties) s.verdict = VBMC_TIES_ONLY;
    else s.verdict = VBMC_SAFE;
}

// A result that timed out holds the exact result of its checked prefix: the
// getters read it and a new call may reuse the handle.
bool usable(vbmc_status st) { return st == VBMC_OK || st == VBMC_ERR_TIMEOUT; }

vbmc_status counters_status(const Counters& c) {
    if (c.err & DERR_PIXELS) return fail(VBMC_ERR_ARG, "pixel list not distinct or out of range");
    if (c.err & DERR_QUEUE) return fail(VBMC_ERR_OOM, "recheck queue overflow: raise caps.queue_cap");
    if (c.err & DERR_TC_WAIT) return fail(VBMC_ERR_DEVICE, "tensor-core pipeline wait timed out");
    return VBMC_OK;
}

vbmc_status finish(vbmc_result* r) {
    if (!r->have_result) return fail(VBMC_ERR_STATE, "no verify call on this result");
    if (r->pending) {
        VB_CUDA(cudaStreamSynchronize(r->last_stream));
        r->pending = false;
        float ms = 0.f, ms_p = 0.f, ms_s = 0.f;
        cudaEventElapsedTime(&ms, r->ev0, r->ev1);
        cudaEventElapsedTime(&ms_p, r->ev0, r->ev_pro);
        cudaEventElapsedTime(&ms_s, r->ev_pro, r->ev_scr);
        float mp[4] = {0.f, 0.f, 0.f, 0.f};
        cudaEventElapsedTime(&mp[0], r->ev_scr, r->ev_split);
        cudaEventElapsedTime(&mp[1], r->ev_split, r->ev_f32);
        cudaEventElapsedTime(&mp[2], r->ev_f32, r->ev_df);
        cudaEventElapsedTime(&mp[3], r->ev_df, r->ev1);
        (void)cudaGetLastError();  // timing is informative only
        fill_summary(r, *r->h_cnt, ms, ms_p, ms_s, mp);
        r->last_status = counters_status(*r->h_cnt);
        if (r->last_status == VBMC_OK && r->sum.checked_hi < r->hi)
            r->last_status = fail(VBMC_ERR_TIMEOUT, "time budget ran out: the summary covers [lo, checked_hi)");
    }
    return r->last_status;
}

}  // namespace

extern "C" vbmc_status vbmc_verify_query_device(vbmc_net* net, const uint8_t* d_image, int32_t s,
                                                const int32_t* d_pixels, int32_t k, uint64_t lo,
                                                uint64_t hi, const vbmc_options* opt,
                                                vbmc_result* res, void* stream) {
    if (!net || !res || !d_image || (!d_pixels && s > 0) || !opt)
        return fail(VBMC_ERR_ARG, "null argument");
    if (res->net != net) return fail(VBMC_ERR_ARG, "result belongs to another net");
    if (res->pending) {
        vbmc_status st = finish(res);
        if (!usable(st)) return st;
    }
    uint64_t n, h;
    vbmc_status st = check_query_shape(res, s, k, lo, hi, opt, &n, &h);
    if (st != VBMC_OK) return st;
    res->image.clear();
    res->pixels.clear();
    return enqueue(net, res, d_image, d_pixels, s, k, lo, h, n, *opt, (cudaStream_t)stream);
}

extern "C" vbmc_status vbmc_verify_query(vbmc_net* net, const vbmc_query* q, const vbmc_options* opt,
                                         vbmc_result* res, void* stream) {
    if (!net || !q || !res || !opt || !q->image || (!q->pixels && q->s > 0))
        return fail(VBMC_ERR_ARG, "null argument");
    if (res->net != net) return fail(VBMC_ERR_ARG, "result belongs to another net");
    if (res->pending) {
        vbmc_status st = finish(res);
        if (!usable(st)) return st;
    }
    uint64_t n, h;
    vbmc_status st = check_query_shape(res, q->s, q->k, q->lo, q->hi, opt, &n, &h);
    if (st != VBMC_OK) return st;
    const int H0 = net->v.dims[0];
    for (int p = 0; p < q->s; ++p) {
        if (q->pixels[p] < 0 || q->pixels[p] >= H0) return fail(VBMC_ERR_ARG, "pixel index out of range");
        for (int r = 0; r < p; ++r)
            if (q->pixels[r] == q->pixels[p]) return fail(VBMC_ERR_ARG, "duplicate pixel index");
    }
    cudaStream_t stq = (cudaStream_t)stream;
    VB_CUDA(cudaMemcpyAsync(res->d_image, q->image, H0, cudaMemcpyHostToDevice, stq));
    if (q->s > 0)
        VB_CUDA(cudaMemcpyAsync(res->d_pix_in, q->pixels, sizeof(int32_t) * q->s,
                                cudaMemcpyHostToDevice, stq));
    QueryExtra x;
    st = query_extra(*q, &x);
    if (st != VBMC_OK) return st;
    st = enqueue(net, res, res->d_image, res->d_pix_in, q->s, q->k, q->lo, h, n, *opt, stq, x);
    if (st != VBMC_OK) return st;
    res->image.assign(q->image, q->image + H0);
    res->pixels.assign(q->pixels, q->pixels + q->s);
    return finish(res);
}

extern "C" vbmc_status vbmc_result_summary(vbmc_result* res, vbmc_summary* out) {
    if (!res || !out) return fail(VBMC_ERR_ARG, "null argument");
    vbmc_status st = finish(res);
    *out = res->sum;
    return st;
}

extern "C" vbmc_status vbmc_get_witness(vbmc_result* res, uint64_t* index, int32_t* steps,
                                        uint8_t* image, double* margin) {
    if (!res) return fail(VBMC_ERR_ARG, "null argument");
    vbmc_status st = finish(res);
    if (!usable(st)) return st;
    const uint64_t t = res->sum.first_witness;
    if (index) *index = t;
    if (t == VBMC_NO_WITNESS) return VBMC_OK;
    const int s = res->s, k = res->k, R = 2 * k + 1;
    std::vector<int> d(s);
    uint64_t tt = t;
    for (int p = s - 1; p >= 0; --p) {
        d[p] = (int)(tt % R);
        tt /= R;
    }
    if (steps)
        for (int p = 0; p < s; ++p) steps[p] = d[p] - k;
    if (image) {
        const int H0 = res->net->v.dims[0];
        std::vector<uint8_t> img(H0);
        std::vector<int32_t> pix(s);
        if (!res->image.empty()) {
            img = res->image;
            pix = res->pixels;
        } else {
            VB_CUDA(cudaMemcpy(img.data(), res->hq.image ? res->hq.image : res->d_image, H0,
                               cudaMemcpyDeviceToHost));
            VB_CUDA(cudaMemcpy(pix.data(), res->hq.pix, sizeof(int) * s, cudaMemcpyDeviceToHost));
        }
        for (int p = 0; p < s; ++p) {
            int v = img[pix[p]] + d[p] - k;
            img[pix[p]] = (uint8_t)std::min(255, std::max(0, v));
        }
        std::memcpy(image, img.data(), H0);
    }
    if (margin) {
        launch_margin64(res->net->v, res->d_q, t, res->d_margin, res->last_stream);
        VB_CUDA(cudaGetLastError());
        VB_CUDA(cudaMemcpyAsync(margin, res->d_margin, sizeof(double), cudaMemcpyDeviceToHost,
                                res->last_stream));
        VB_CUDA(cudaStreamSynchronize(res->last_stream));
    }
    return VBMC_OK;
}

extern "C" vbmc_status vbmc_get_coverage(vbmc_result* res, uint32_t* flip, size_t flip_words,
                                         uint32_t* flip_tie, uint32_t* ss, size_t ss_words,
                                         uint32_t* ss_tie, double* covered_fraction) {
    if (!res) return fail(VBMC_ERR_ARG, "null argument");
    vbmc_status st = finish(res);
    if (!usable(st)) return st;
    if (!res->opt.coverage) return fail(VBMC_ERR_STATE, "coverage was off for the last call");
    const NetView& v = res->net->v;
    if ((flip || flip_tie) && flip_words < (size_t)v.flip_words)
        return fail(VBMC_ERR_ARG, "flip buffer too small");
    if ((ss || ss_tie || covered_fraction) && ss && ss_words < (size_t)v.ss_words)
        return fail(VBMC_ERR_ARG, "ss buffer too small");
    if (flip) VB_CUDA(cudaMemcpy(flip, res->hq.flip, 4ull * v.flip_words, cudaMemcpyDeviceToHost));
    if (flip_tie)
        VB_CUDA(cudaMemcpy(flip_tie, res->hq.flip_tie, 4ull * v.flip_words, cudaMemcpyDeviceToHost));
    std::vector<uint32_t> tmp;
    uint32_t* ssh = ss;
    if (!ssh && covered_fraction) {
        tmp.resize(v.ss_words);
        ssh = tmp.data();
    }
    if (ssh) VB_CUDA(cudaMemcpy(ssh, res->hq.ss, 4ull * v.ss_words, cudaMemcpyDeviceToHost));
    if (ss_tie) VB_CUDA(cudaMemcpy(ss_tie, res->hq.ss_tie, 4ull * v.ss_words, cudaMemcpyDeviceToHost));
    if (covered_fraction) {
        // Eq. 3: neurons in at least one SS-covered pair over all non-input neurons.
        std::vector<char> cov(v.total, 0);
        for (int l = 1; l < v.L; ++l) {
            const int Hl = v.dims[l], Hn = v.dims[l + 1];
            for (int j = 0; j < Hl; ++j)
                for (int i = 0; i < Hn; ++i) {
                    const unsigned long long b = v.ssoff[l] + (unsigned long long)j * Hn + i;
                    if ((ssh[b >> 5] >> (b & 31)) & 1u) {
                        cov[v.noff[l] + j] = 1;
                        cov[v.noff[l + 1] + i] = 1;
                    }
                }
        }
        int c = 0;
        for (char x : cov) c += x;
        *covered_fraction = (double)c / (double)v.total;
    }
    return VBMC_OK;
}

extern "C" vbmc_status vbmc_get_verdict_bitmap(vbmc_result* res, uint32_t* words, size_t n_words) {
    if (!res || !words) return fail(VBMC_ERR_ARG, "null argument");
    vbmc_status st = finish(res);
    if (!usable(st)) return st;
    if (!res->opt.bitmap) return fail(VBMC_ERR_STATE, "bitmap was off for the last call");
    const size_t need = (size_t)((res->hi + 31) / 32);
    if (n_words < need) return fail(VBMC_ERR_ARG, "bitmap buffer too small");
    VB_CUDA(cudaMemcpy(words, res->hq.bitmap, 4 * need, cudaMemcpyDeviceToHost));
    return VBMC_OK;
}

extern "C" vbmc_status vbmc_get_ties(vbmc_result* res, uint64_t* idx, size_t cap, uint64_t* n_ties) {
    if (!res) return fail(VBMC_ERR_ARG, "null argument");
    vbmc_status st = finish(res);
    if (!usable(st)) return st;
    const uint64_t n = res->sum.n_ties;
    if (n_ties) *n_ties = n;
    const size_t kept = (size_t)std::min<uint64_t>(n, res->caps.ties_cap);
    if (idx && cap) {
        std::vector<uint64_t> t(kept);
        if (kept) VB_CUDA(cudaMemcpy(t.data(), res->hq.ties, 8 * kept, cudaMemcpyDeviceToHost));
        std::sort(t.begin(), t.end());
        std::memcpy(idx, t.data(), 8 * std::min(cap, kept));
    }
    return VBMC_OK;
}

extern "C" vbmc_status vbmc_verify_batch(vbmc_net* net, const vbmc_query* queries, int32_t nq,
                                         const vbmc_options* opt, vbmc_result* const* results,
                                         void* stream) {
    if (!net || (!queries && nq > 0) || !opt || (!results && nq > 0))
        return fail(VBMC_ERR_ARG, "null argument");
    if (nq == 0) return VBMC_OK;
    BatchArena* ar = results[0] ? results[0]->arena : nullptr;
    bool together = ar && ar->nq >= nq;
    for (int i = 0; i < nq && together; ++i)
        together = results[i] && results[i]->arena == ar && results[i]->slot == i && results[i]->net == net;
    // results not created together, or a precision whose screen serves one query
    // at a time (the wide-layer path): one query after another
    if (!together || opt->precision == VBMC_PREC_FP8 ||
        ((opt->precision == VBMC_PREC_BF16 || opt->precision == VBMC_PREC_FP16) && !tc_supported(net->v, opt->precision))) {
        for (int i = 0; i < nq; ++i) {
            vbmc_status st = vbmc_verify_query(net, &queries[i], opt, results[i], stream);
            if (st != VBMC_OK) return st;
        }
        return VBMC_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (opt->graph) {
        // capture on the batch's own stream, after everything already on the caller's
        VB_CUDA(cudaEventRecord(ar->gev, st));
        VB_CUDA(cudaStreamWaitEvent(ar->gstream, ar->gev, 0));
        st = ar->gstream;
    }
    const NetView& v = net->v;
    const int H0 = v.dims[0];
    // validate, stage images and pixel lists in one buffer, build the views
    std::vector<uint8_t> stage(ar->stage_stride * (size_t)nq, 0);
    std::vector<QueryView> hq((size_t)nq);
    std::vector<uint64_t> nsp((size_t)nq);
    for (int i = 0; i < nq; ++i) {
        const vbmc_query& q = queries[i];
        vbmc_result* r = results[i];
        if (r->pending) {
            vbmc_status fs = finish(r);
            if (!usable(fs)) return fs;
        }
        if (!q.image || (!q.pixels && q.s > 0)) return fail(VBMC_ERR_ARG, "null query buffer");
        uint64_t n, h;
        vbmc_status cs = check_query_shape(r, q.s, q.k, q.lo, q.hi, opt, &n, &h);
        if (cs != VBMC_OK) return cs;
        for (int p = 0; p < q.s; ++p) {
            if (q.pixels[p] < 0 || q.pixels[p] >= H0) return fail(VBMC_ERR_ARG, "pixel index out of range");
            for (int rr = 0; rr < p; ++rr)
                if (q.pixels[rr] == q.pixels[p]) return fail(VBMC_ERR_ARG, "duplicate pixel index");
        }
        uint8_t* slot = stage.data() + ar->stage_stride * (size_t)i;
        std::memcpy(slot, q.image, (size_t)H0);
        std::memcpy(slot + ((H0 + 3) & ~3), q.pixels, sizeof(int32_t) * (size_t)q.s);
        const uint8_t* d_img = ar->d_stage + ar->stage_stride * (size_t)i;
        const int* d_pix = reinterpret_cast<const int*>(d_img + ((H0 + 3) & ~3));
        QueryExtra x;
        const vbmc_status xs = query_extra(q, &x);
        if (xs != VBMC_OK) return xs;
        hq[i] = make_view(r, d_img, d_pix, q.s, q.k, q.lo, h, n, *opt, i, x);
        nsp[i] = n;
    }
    std::vector<unsigned long long> tp = tile_prefix(v, opt->precision, hq.data(), nq);
    // run order: the passes see the views in schedule order (each view still
    // points at its own result's counters and buffers; queue entries index
    // the run order)
    std::vector<int> perm((size_t)nq);
    for (int i = 0; i < nq; ++i) perm[i] = i;
    if (opt->schedule == VBMC_SCHED_SMALL_FIRST)
        std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
            return hq[a].hi - hq[a].lo < hq[b].hi - hq[b].lo;
        });
    std::vector<QueryView> hrun((size_t)nq);
    for (int j = 0; j < nq; ++j) {
        hrun[j] = hq[perm[j]];
        hrun[j].qid = j;
    }
    // waves: the smallest-first schedule runs the queries in up to 8 waves of
    // about equal work, each its own chain of passes, so the queries of an early
    // wave are final when that wave ends (and each wave's rechecks queue alone)
    std::vector<int> wave_at{0};
    if (opt->schedule == VBMC_SCHED_SMALL_FIRST) {
        unsigned long long total = 0, acc = 0;
        for (int j = 0; j < nq; ++j) total += hrun[j].hi - hrun[j].lo;
        const int W = std::min(8, nq);
        for (int j = 0; j < nq; ++j) {
            acc += hrun[j].hi - hrun[j].lo;
            const int w = (int)wave_at.size();
            if (w < W && j + 1 < nq && (double)acc >= (double)total * w / W) wave_at.push_back(j + 1);
        }
    }
    wave_at.push_back(nq);
    const int n_waves = (int)wave_at.size() - 1;
    // per-wave tile prefixes, back to back: wave w's starts at tp_at[w]
    std::vector<unsigned long long> tpall;
    std::vector<size_t> tp_at;
    std::vector<unsigned long long> wave_tiles;
    for (int w = 0; w < n_waves; ++w) {
        const int j0 = wave_at[w], j1 = wave_at[w + 1];
        const std::vector<unsigned long long> t = tile_prefix(v, opt->precision, hrun.data() + j0, j1 - j0);
        tp_at.push_back(tpall.size());
        tpall.insert(tpall.end(), t.begin(), t.end());
        wave_tiles.push_back(t.back());
    }
    VB_CUDA(cudaMemcpyAsync(ar->d_stage, stage.data(), stage.size(), cudaMemcpyHostToDevice, st));
    VB_CUDA(cudaMemcpyAsync(ar->d_qs, hq.data(), sizeof(QueryView) * (size_t)nq, cudaMemcpyHostToDevice, st));
    VB_CUDA(cudaMemcpyAsync(ar->d_qs_run, hrun.data(), sizeof(QueryView) * (size_t)nq,
                            cudaMemcpyHostToDevice, st));
    VB_CUDA(cudaMemcpyAsync(ar->d_tp, tpall.data(), sizeof(unsigned long long) * tpall.size(),
                            cudaMemcpyHostToDevice, st));
    auto run_waves = [&](bool capturing) -> vbmc_status {
        for (int w = 0; w < n_waves; ++w) {
            const int j0 = wave_at[w], j1 = wave_at[w + 1];
            // pass times are those of the first wave
            const cudaEvent_t evs[7] = {w == 0 ? ar->ev[0] : ar->evw, w == 0 ? ar->ev[1] : ar->evw,
                                        w == 0 ? ar->ev[2] : ar->evw, w == n_waves - 1 ? ar->ev[3] : ar->evw,
                                        w == 0 ? ar->ev[4] : ar->evw, w == 0 ? ar->ev[5] : ar->evw,
                                        w == 0 ? ar->ev[6] : ar->evw};
            vbmc_status ws = enqueue_passes(net, ar->d_qs_run + j0, hrun.data() + j0, j1 - j0,
                                            ar->d_tp + tp_at[w], wave_tiles[w], ar->d_qcount, ar->d_queue,
                                            ar->queue_cap, evs, *opt, st, capturing, STAGE_ALL, nullptr, nullptr,
                                            ar->d_claim);
            if (ws != VBMC_OK) return ws;
        }
        return VBMC_OK;
    };
    vbmc_status sst;
    if (opt->graph) {
        // the passes as one CUDA graph (the host-to-device copies above stay
        // outside); captured and instantiated once per batch shape, then relaunched
        std::string sig = std::to_string(nq) + ":" + std::to_string(opt->precision) + ":" +
                          std::to_string(opt->coverage) + ":" + std::to_string(opt->bitmap) + ":" +
                          std::to_string(opt->schedule);
        for (int j = 0; j < nq; ++j) {
            const QueryView& h = hrun[j];
            sig += "|" + std::to_string(h.s) + "," + std::to_string(h.k) + "," + std::to_string(h.lo) + "," +
                   std::to_string(h.hi) + "," + std::to_string(h.filter) + "," + std::to_string(h.l2max) + "," +
                   std::to_string(h.prop) + "," + std::to_string(perm[j]);
        }
        if (!ar->gexec || ar->gsig != sig) {
            if (ar->gexec) cudaGraphExecDestroy(ar->gexec);
            ar->gexec = nullptr;
            ar->gsig.clear();
            cudaGraph_t g = nullptr;
            VB_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            sst = run_waves(true);
            cudaError_t ce = cudaStreamEndCapture(st, &g);
            if (sst != VBMC_OK) {
                if (g) cudaGraphDestroy(g);
                return sst;
            }
            if (ce != cudaSuccess) return fail(VBMC_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&ar->gexec, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) {
                ar->gexec = nullptr;
                return fail(VBMC_ERR_CUDA, std::string("graph: ") + cudaGetErrorString(ce));
            }
            ar->gsig = sig;
        }
        // the thresholds of Eq. 11 live in the views (copied above), not in the graph
        cudaError_t ce = cudaGraphLaunch(ar->gexec, st);
        if (ce != cudaSuccess) return fail(VBMC_ERR_CUDA, std::string("graph: ") + cudaGetErrorString(ce));
    } else {
        sst = run_waves(false);
        if (sst != VBMC_OK) return sst;
    }
    VB_CUDA(cudaMemcpyAsync(ar->h_cnt, ar->d_cnt, sizeof(Counters) * (size_t)nq, cudaMemcpyDeviceToHost, st));
    VB_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f, ms_p = 0.f, ms_s = 0.f;
    cudaEventElapsedTime(&ms, ar->ev[0], ar->ev[3]);
    cudaEventElapsedTime(&ms_p, ar->ev[0], ar->ev[1]);
    cudaEventElapsedTime(&ms_s, ar->ev[1], ar->ev[2]);
    float mp[4] = {0.f, 0.f, 0.f, 0.f};
    if (n_waves == 1) {
        cudaEventElapsedTime(&mp[0], ar->ev[2], ar->ev[4]);
        cudaEventElapsedTime(&mp[1], ar->ev[4], ar->ev[5]);
        cudaEventElapsedTime(&mp[2], ar->ev[5], ar->ev[6]);
        cudaEventElapsedTime(&mp[3], ar->ev[6], ar->ev[3]);
    }
    (void)cudaGetLastError();  // timing is informative only
    vbmc_status result = VBMC_OK;
    for (int i = 0; i < nq; ++i) {
        vbmc_result* r = results[i];
        const vbmc_query& q = queries[i];
        r->last_stream = st;
        r->pending = false;
        r->have_result = true;
        r->s = q.s;
        r->k = q.k;
        r->lo = q.lo;
        r->hi = hq[i].hi;
        r->n_space = nsp[i];
        r->opt = *opt;
        r->image.assign(q.image, q.image + H0);
        r->pixels.assign(q.pixels, q.pixels + q.s);
        r->hq.image = hq[i].image;
        r->tile_pts = 0;  // batches check every tile (no budget)
        fill_summary(r, ar->h_cnt[i], ms, ms_p, ms_s, mp);
        r->last_status = counters_status(ar->h_cnt[i]);
        if (r->last_status != VBMC_OK && result == VBMC_OK) result = r->last_status;
    }
    return result;
}

namespace vbmc {
vbmc_status launch_enum_pairs(const NetView& v, const QueryView& q, const vbmc_cover_params* params,
                              const vbmc_pair_masks* out, unsigned long long* d_npoints, cudaStream_t st);
}

extern "C" vbmc_status vbmc_enum_coverage(vbmc_net* net, const vbmc_query* q, const vbmc_cover_params* params,
                                          const vbmc_pair_masks* out, vbmc_result* res, uint64_t* n_points,
                                          void* stream) {
    if (!net || !q || !params || !out || !res || !q->image || (!q->pixels && q->s > 0))
        return fail(VBMC_ERR_ARG, "null argument");
    if (res->net != net) return fail(VBMC_ERR_ARG, "result belongs to another net");
    if (res->pending) {
        vbmc_status st = finish(res);
        if (!usable(st)) return st;
    }
    uint64_t n, h;
    vbmc_status st = check_query_shape(res, q->s, q->k, q->lo, q->hi, nullptr, &n, &h);
    if (st != VBMC_OK) return st;
    const int H0 = net->v.dims[0];
    for (int p = 0; p < q->s; ++p) {
        if (q->pixels[p] < 0 || q->pixels[p] >= H0) return fail(VBMC_ERR_ARG, "pixel index out of range");
        for (int r = 0; r < p; ++r)
            if (q->pixels[r] == q->pixels[p]) return fail(VBMC_ERR_ARG, "duplicate pixel index");
    }
    QueryExtra x;
    st = query_extra(*q, &x);
    if (st != VBMC_OK) return st;
    cudaStream_t sq = (cudaStream_t)stream;
    VB_CUDA(cudaMemcpyAsync(res->d_image, q->image, H0, cudaMemcpyHostToDevice, sq));
    if (q->s > 0)
        VB_CUDA(cudaMemcpyAsync(res->d_pix_in, q->pixels, sizeof(int32_t) * q->s, cudaMemcpyHostToDevice, sq));
    vbmc_options none{};
    const QueryView qv = make_view(res, res->d_image, res->d_pix_in, q->s, q->k, q->lo, h, n, none, 0, x);
    // the result's point counter carries the count; its verify state is gone
    res->have_result = false;
    unsigned long long* dn = &res->d_cnt->n_points;
    VB_CUDA(cudaMemsetAsync(dn, 0, sizeof(unsigned long long), sq));
    st = launch_enum_pairs(net->v, qv, params, out, dn, sq);
    if (st != VBMC_OK) return st;
    unsigned long long hn = 0;
    VB_CUDA(cudaMemcpyAsync(&hn, dn, sizeof(hn), cudaMemcpyDeviceToHost, sq));
    VB_CUDA(cudaStreamSynchronize(sq));
    if (n_points) *n_points = hn;
    return VBMC_OK;
}

extern "C" vbmc_status vbmc_wide_trace(vbmc_net* net, const vbmc_query* q, int32_t precision, int32_t n_points,
                                       float* vals, float* nre, vbmc_result* res, void* stream) {
    if (!net || !q || !res || !vals || !nre) return fail(VBMC_ERR_ARG, "null argument");
    const NetView& v = net->v;
    const bool wide = wide_type(precision) >= 0 && wide_supported(v) &&
                      (precision == VBMC_PREC_FP8 || !tc_supported(v, precision));
    if (!wide) return fail(VBMC_ERR_UNSUPPORTED, "this net and precision do not take the wide-layer path");
    const uint64_t n = space_size(q->s, q->k);
    if (n_points < 1 || (uint64_t)n_points > n) return fail(VBMC_ERR_ARG, "n_points outside [1, R^s]");
    const size_t nv = (size_t)(v.L - 1) * n_points * v.hmax, nn = (size_t)(v.L - 1) * n_points * 3;
    float *dvals = nullptr, *dnre = nullptr;
    if (cudaMalloc(&dvals, sizeof(float) * nv) != cudaSuccess || cudaMalloc(&dnre, sizeof(float) * nn) != cudaSuccess) {
        cudaFree(dvals);
        return fail(VBMC_ERR_OOM, "trace buffers");
    }
    cudaMemset(dvals, 0, sizeof(float) * nv);
    cudaMemset(dnre, 0, sizeof(float) * nn);
    WideTrace t;
    t.vals = dvals;
    t.nre = dnre;
    t.n = n_points;
    t.hmax = v.hmax;
    wide_set_trace(&t);
    vbmc_query qq = *q;
    qq.lo = 0;
    qq.hi = (uint64_t)n_points;
    vbmc_options o{};
    o.precision = precision;
    vbmc_status st = vbmc_verify_query(net, &qq, &o, res, stream);
    if (st == VBMC_OK) st = finish(res);
    wide_set_trace(nullptr);
    if (st == VBMC_OK &&
        (cudaMemcpy(vals, dvals, sizeof(float) * nv, cudaMemcpyDeviceToHost) != cudaSuccess ||
         cudaMemcpy(nre, dnre, sizeof(float) * nn, cudaMemcpyDeviceToHost) != cudaSuccess))
        st = fail(VBMC_ERR_CUDA, "trace copy");
    cudaFree(dvals);
    cudaFree(dnre);
    return st;
}

extern "C" vbmc_status vbmc_search_query(vbmc_net* net, const vbmc_query* q, int32_t n_tiles,
                                         const int32_t* order, const vbmc_options* opt, vbmc_result* res,
                                         vbmc_search_out* out, void* stream) {
    if (!net || !q || !res || !opt || !order || !q->image || (!q->pixels && q->s > 0))
        return fail(VBMC_ERR_ARG, "null argument");
    if (res->net != net) return fail(VBMC_ERR_ARG, "result belongs to another net");
    if (n_tiles < 1) return fail(VBMC_ERR_ARG, "n_tiles must be positive");
    if (res->pending) {
        vbmc_status st = finish(res);
        if (!usable(st)) return st;
    }
    uint64_t n, h;
    vbmc_status st = check_query_shape(res, q->s, q->k, 0, 0, opt, &n, &h);
    if (st != VBMC_OK) return st;
    if (q->lo != 0 || (q->hi != 0 && q->hi != n))
        return fail(VBMC_ERR_ARG, "a search covers the whole space: lo and hi must be 0");
    std::vector<char> seen((size_t)n_tiles, 0);
    for (int i = 0; i < n_tiles; ++i) {
        if (order[i] < 0 || order[i] >= n_tiles || seen[order[i]])
            return fail(VBMC_ERR_ARG, "order is not a permutation of the tiles");
        seen[order[i]] = 1;
    }
    const int H0 = net->v.dims[0];
    for (int p = 0; p < q->s; ++p) {
        if (q->pixels[p] < 0 || q->pixels[p] >= H0) return fail(VBMC_ERR_ARG, "pixel index out of range");
        for (int r = 0; r < p; ++r)
            if (q->pixels[r] == q->pixels[p]) return fail(VBMC_ERR_ARG, "duplicate pixel index");
    }
    cudaStream_t sq = (cudaStream_t)stream;
    VB_CUDA(cudaMemcpyAsync(res->d_image, q->image, H0, cudaMemcpyHostToDevice, sq));
    if (q->s > 0)
        VB_CUDA(cudaMemcpyAsync(res->d_pix_in, q->pixels, sizeof(int32_t) * q->s, cudaMemcpyHostToDevice, sq));
    const unsigned long long cap = std::max<uint64_t>(1, res->caps.queue_cap);
    // set-up once over the whole space: counters, cleared masks and bitmap, tables
    QueryExtra x;
    st = query_extra(*q, &x);
    if (st != VBMC_OK) return st;
    QueryView qv = make_view(res, res->d_image, res->d_pix_in, q->s, q->k, 0, n, n, *opt, 0, x);
    std::vector<unsigned long long> tp = tile_prefix(net->v, opt->precision, &qv, 1);
    VB_CUDA(cudaMemcpyAsync(res->d_q, &qv, sizeof(QueryView), cudaMemcpyHostToDevice, sq));
    const cudaEvent_t ev_set[7] = {res->ev0,    res->ev_pro, res->ev_pro, res->ev_pro,
                                   res->ev_pro, res->ev_pro, res->ev_pro};
    st = enqueue_passes(net, res->d_q, &qv, 1, res->d_tp, tp[1], res->d_qcount, res->d_queue, cap, ev_set,
                        *opt, sq, false, STAGE_SETUP, &res->ww, res->have_tw ? &res->tw : nullptr);
    if (st != VBMC_OK) return st;
    const cudaEvent_t ev_tile[7] = {res->ev_scr, res->ev_scr, res->ev_scr, res->ev1,
                                    res->ev_scr, res->ev_scr, res->ev_scr};
    const uint64_t tsize = (n + n_tiles - 1) / n_tiles;
    vbmc_search_out so{0, -1, 0, 0.0};
    vbmc_status run = VBMC_OK;
    bool any_tile = false;
    for (int i = 0; i < n_tiles; ++i) {
        const uint64_t lo = (uint64_t)order[i] * tsize;
        const uint64_t hi = std::min<uint64_t>(n, lo + tsize);
        so.tiles_checked += 1;
        if (lo >= hi) continue;
        qv.lo = lo;
        qv.hi = hi;
        tp = tile_prefix(net->v, opt->precision, &qv, 1);
        VB_CUDA(cudaMemcpyAsync(res->d_q, &qv, sizeof(QueryView), cudaMemcpyHostToDevice, sq));
        VB_CUDA(cudaMemcpyAsync(res->d_tp, tp.data(), sizeof(unsigned long long) * 2, cudaMemcpyHostToDevice,
                                sq));
        st = enqueue_passes(net, res->d_q, &qv, 1, res->d_tp, tp[1], res->d_qcount, res->d_queue, cap, ev_tile,
                            *opt, sq, false, STAGE_PASSES, &res->ww, res->have_tw ? &res->tw : nullptr);
        if (st != VBMC_OK) return st;
        any_tile = true;
        VB_CUDA(cudaMemcpyAsync(res->h_cnt, res->d_cnt, sizeof(Counters), cudaMemcpyDeviceToHost, sq));
        VB_CUDA(cudaStreamSynchronize(sq));
        so.points_checked += hi - lo;
        run = counters_status(*res->h_cnt);
        if (run != VBMC_OK) break;
        if (res->h_cnt->n_adv > 0) {
            so.witness_tile = order[i];
            break;
        }
    }
    if (qv.filter) so.points_checked = res->h_cnt->n_points;  // the passes counted what passed the filter
    if (!any_tile) {
        VB_CUDA(cudaEventRecord(res->ev1, sq));
        VB_CUDA(cudaMemcpyAsync(res->h_cnt, res->d_cnt, sizeof(Counters), cudaMemcpyDeviceToHost, sq));
    }
    VB_CUDA(cudaStreamSynchronize(sq));
    float ms = 0.f, ms_p = 0.f;
    cudaEventElapsedTime(&ms, res->ev0, res->ev1);
    cudaEventElapsedTime(&ms_p, res->ev0, res->ev_pro);
    so.ms_to_witness = ms;
    res->last_stream = sq;
    res->pending = false;
    res->have_result = true;
    res->s = q->s;
    res->k = q->k;
    res->lo = 0;
    res->hi = n;
    res->n_space = n;
    res->opt = *opt;
    res->image.assign(q->image, q->image + H0);
    res->pixels.assign(q->pixels, q->pixels + q->s);
    res->tile_pts = 0;  // the tile search checks whole tiles (no budget)
    fill_summary(res, *res->h_cnt, ms, ms_p, 0.f);
    res->sum.n_points = so.points_checked;
    res->sum.ms_to_verdict = ms;
    if (run == VBMC_OK) run = counters_status(*res->h_cnt);
    if (run != VBMC_OK) res->sum.verdict = VBMC_PARTIAL;
    res->last_status = run;
    if (out) *out = so;
    return run;
}

extern "C" vbmc_status vbmc_tile_counts(vbmc_result* res, int32_t n_tiles, uint64_t* counts) {
    if (!res || !counts) return fail(VBMC_ERR_ARG, "null argument");
    if (n_tiles < 1) return fail(VBMC_ERR_ARG, "n_tiles must be positive");
    vbmc_status st = finish(res);
    if (!usable(st)) return st;
    if (!res->opt.bitmap) return fail(VBMC_ERR_STATE, "bitmap was off for the last call");
    if (res->lo != 0 || res->hi != res->n_space)
        return fail(VBMC_ERR_STATE, "the last call did not cover the whole space");
    if (n_tiles > VBMC_MAX_TILES) return fail(VBMC_ERR_ARG, "n_tiles above VBMC_MAX_TILES");
    unsigned long long* d = res->d_tiles;
    launch_tile_counts(res->hq.bitmap, res->n_space, n_tiles, d, res->last_stream);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(counts, d, sizeof(unsigned long long) * n_tiles, cudaMemcpyDeviceToHost,
                            res->last_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(res->last_stream);
    if (e != cudaSuccess) return fail(VBMC_ERR_CUDA, cudaGetErrorString(e));
    return VBMC_OK;
}

// ------------------------------------------------------------------ autotuning

namespace {

__global__ void k_fill_queue(QEntry* e, unsigned long long n, unsigned long long stride) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    QEntry x;
    x.t = i * stride;
    x.q = 0;
    x.pad = 0;
    e[i] = x;
}

std::string tune_key(const vbmc_net* net) {
    cudaDeviceProp p{};
    cudaGetDeviceProperties(&p, net->device);
    std::string k = "passes=fp32,df;dims=";
    for (int l = 0; l <= net->v.L; ++l) k += (l ? "x" : "") + std::to_string(net->v.dims[l]);
    k += ";act=" + std::to_string(net->v.act) + ";sm=" + std::to_string(net->n_sm) +
         ";cc=" + std::to_string(p.major * 10 + p.minor);
    return k;
}

bool json_int(const std::string& line, const char* name, int* v) {
    const std::string pat = std::string("\"") + name + "\": ";
    const size_t i = line.find(pat);
    if (i == std::string::npos) return false;
    *v = std::atoi(line.c_str() + i + pat.size());
    return true;
}

// One JSON object per line: {"key": "...", "simt_range": v, ...}.
bool cache_lookup(const char* path, const std::string& key, vbmc_tuning* t) {
    FILE* f = path ? std::fopen(path, "r") : nullptr;
    if (!f) return false;
    char buf[1024];
    bool hit = false;
    const std::string pat = "\"key\": \"" + key + "\"";
    while (!hit && std::fgets(buf, sizeof(buf), f)) {
        const std::string line(buf);
        if (line.find(pat) == std::string::npos) continue;
        hit = json_int(line, "simt_range", &t->simt_range) &&
              json_int(line, "simt_range_ctas", &t->simt_range_ctas) &&
              json_int(line, "simt_gather", &t->simt_gather) &&
              json_int(line, "simt_gather_ctas", &t->simt_gather_ctas) &&
              json_int(line, "df_ctas", &t->df_ctas);
    }
    std::fclose(f);
    return hit;
}

bool cache_store(const char* path, const std::string& key, const vbmc_tuning& t) {
    std::vector<std::string> keep;
    const std::string pat = "\"key\": \"" + key + "\"";
    if (FILE* f = std::fopen(path, "r")) {
        char buf[1024];
        while (std::fgets(buf, sizeof(buf), f)) {
            std::string line(buf);
            if (line.find(pat) == std::string::npos && line.find("\"key\"") != std::string::npos)
                keep.push_back(line);
        }
        std::fclose(f);
    }
    char row[1024];
    std::snprintf(row, sizeof(row),
                  "{\"key\": \"%s\", \"simt_range\": %d, \"simt_range_ctas\": %d, \"simt_gather\": %d, "
                  "\"simt_gather_ctas\": %d, \"df_ctas\": %d, \"ms_range\": %.4f, \"ms_gather\": %.4f, "
                  "\"ms_df\": %.4f}\n",
                  key.c_str(), t.simt_range, t.simt_range_ctas, t.simt_gather, t.simt_gather_ctas, t.df_ctas,
                  t.ms_range, t.ms_gather, t.ms_df);
    keep.push_back(row);
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    for (const std::string& l : keep) std::fputs(l.c_str(), f);
    std::fclose(f);
    return std::rename(tmp.c_str(), path) == 0;
}

void apply_tuning(vbmc_net* net, const vbmc_tuning& t) {
    net->v.simt_var_range = t.simt_range;
    net->v.simt_ctas_range = t.simt_range_ctas;
    net->v.simt_var_gather = t.simt_gather;
    net->v.simt_ctas_gather = t.simt_gather_ctas;
    net->v.df_ctas = t.df_ctas;
}

}  // namespace

extern "C" vbmc_status vbmc_set_tuning(vbmc_net* net, const vbmc_tuning* t) {
    if (!net || !t) return fail(VBMC_ERR_ARG, "null argument");
    apply_tuning(net, *t);
    return VBMC_OK;
}

extern "C" vbmc_status vbmc_autotune(vbmc_net* net, const char* cache_path, vbmc_tuning* out) {
    if (!net) return fail(VBMC_ERR_ARG, "null argument");
    const NetView& v = net->v;
    if (simt_variant_default(v) == 0) return fail(VBMC_ERR_UNSUPPORTED, "layer width above 1024");
    const std::string key = tune_key(net);
    vbmc_tuning t{};
    if (cache_lookup(cache_path, key, &t)) {
        t.from_cache = 1;
        apply_tuning(net, t);
        if (out) *out = t;
        return VBMC_OK;
    }
    // sample box: s <= 4 pixels spread over the input, k so that R^s >= 2^17
    const int H0 = v.dims[0];
    const int s = std::min(4, H0);
    int k = 1;
    while (k < VBMC_MAX_K && space_size(s, k) < (1ull << 17)) ++k;
    const uint64_t n = space_size(s, k);
    std::vector<uint8_t> img((size_t)H0);
    for (int j = 0; j < H0; ++j) img[j] = (uint8_t)((j * 37 + 11) & 255);
    std::vector<int32_t> pix((size_t)s);
    for (int p = 0; p < s; ++p) pix[p] = (int32_t)(((long long)p * H0) / s);
    vbmc_caps caps{n, s, k, 1u << 12, n};
    vbmc_result* r = nullptr;
    vbmc_status st = create_result(net, &caps, nullptr, 0, &r);
    if (st != VBMC_OK) return st;
    struct Guard {
        vbmc_result* r;
        ~Guard() { vbmc_result_free(r); }
    } guard{r};
    const vbmc_options o32{VBMC_PREC_FP32, 1, 0, 0, VBMC_SCHED_GIVEN};
    const vbmc_query q{img.data(), s, pix.data(), k, 0, 0};
    const vbmc_tuning saved{v.simt_var_range, v.simt_ctas_range, v.simt_var_gather, v.simt_ctas_gather,
                            v.df_ctas, 0, 0.0, 0.0, 0.0};
    cudaStream_t sq = nullptr;
    VB_CUDA(cudaStreamCreateWithFlags(&sq, cudaStreamNonBlocking));
    struct SGuard {
        cudaStream_t s;
        ~SGuard() { cudaStreamDestroy(s); }
    } sguard{sq};
    st = vbmc_verify_query(net, &q, &o32, r, sq);  // prologue, tables, warm-up
    if (st != VBMC_OK) return st;
    cudaEvent_t e0, e1;
    VB_CUDA(cudaEventCreate(&e0));
    VB_CUDA(cudaEventCreate(&e1));
    const unsigned long long cap = caps.queue_cap;
    Queue qdf{r->d_queue[2], r->d_qcount + 2, cap};
    Queue q64{r->d_queue[3], r->d_qcount + 3, cap};
    auto time_it = [&](auto&& launch) {
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaMemsetAsync(r->d_qcount + 2, 0, sizeof(unsigned long long) * 2, sq);
            cudaEventRecord(e0, sq);
            launch();
            cudaEventRecord(e1, sq);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
        return best;
    };
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, net->device);
    // FP32 pass over the whole box (range mode) and over the same points queued
    std::vector<unsigned long long> qn{n};
    VB_CUDA(cudaMemsetAsync(r->d_qcount + 1, 0, sizeof(unsigned long long), sq));
    k_fill_queue<<<(unsigned)((n + 255) / 256), 256, 0, sq>>>(r->d_queue[1], n, 1);
    VB_CUDA(cudaMemcpyAsync(r->d_qcount + 1, qn.data(), sizeof(unsigned long long), cudaMemcpyHostToDevice, sq));
    float best_r = 1e30f, best_g = 1e30f;
    for (int var = 1; var <= kSimtVariants; ++var) {
        if (v.hmax > simt_variant_width(var)) continue;
        const size_t sm = simt_variant_smem(var);
        for (int ctas = 1; ctas <= 4; ctas *= 2) {
            if ((size_t)ctas * (sm + 1024) > (size_t)max_smem) continue;
            net->v.simt_var_range = net->v.simt_var_gather = var;
            net->v.simt_ctas_range = net->v.simt_ctas_gather = ctas;
            QueryView qv = make_view(r, r->d_image, r->d_pix_in, s, k, 0, n, n, o32, 0);
            std::vector<unsigned long long> tp = tile_prefix(net->v, VBMC_PREC_FP32, &qv, 1);
            VB_CUDA(cudaMemcpyAsync(r->d_q, &qv, sizeof(QueryView), cudaMemcpyHostToDevice, sq));
            VB_CUDA(cudaMemcpyAsync(r->d_tp, tp.data(), sizeof(unsigned long long) * 2, cudaMemcpyHostToDevice, sq));
            const float mr = time_it([&] {
                launch_screen_simt(net->v, r->d_q, 1, r->d_tp, tp[1], nullptr, nullptr, 0, qdf, 2, net->n_sm, sq);
            });
            const float mg = time_it([&] {
                launch_screen_simt(net->v, r->d_q, 1, nullptr, 0, r->d_queue[1], r->d_qcount + 1, cap, qdf, 2,
                                   net->n_sm, sq);
            });
            if (mr < best_r) {
                best_r = mr;
                t.simt_range = var;
                t.simt_range_ctas = ctas;
            }
            if (mg < best_g) {
                best_g = mg;
                t.simt_gather = var;
                t.simt_gather_ctas = ctas;
            }
        }
    }
    // double-float pass over 8192 queued points spread over the box
    const unsigned long long ndf = std::min<unsigned long long>(8192, n);
    std::vector<unsigned long long> dn{ndf};
    k_fill_queue<<<(unsigned)((ndf + 255) / 256), 256, 0, sq>>>(r->d_queue[1], ndf, n / ndf);
    VB_CUDA(cudaMemcpyAsync(r->d_qcount + 1, dn.data(), sizeof(unsigned long long), cudaMemcpyHostToDevice, sq));
    float best_d = 1e30f;
    for (int per = 2; per <= 16; per *= 2) {
        net->v.df_ctas = per;
        const float md = time_it([&] {
            launch_df(net->v, r->d_q, 1, r->d_queue[1], r->d_qcount + 1, cap, q64, 3, net->n_sm, sq);
        });
        if (md < best_d) {
            best_d = md;
            t.df_ctas = per;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const cudaError_t ce = cudaStreamSynchronize(sq);
    if (ce != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        apply_tuning(net, saved);
        return fail(VBMC_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(ce));
    }
    t.ms_range = best_r;
    t.ms_gather = best_g;
    t.ms_df = best_d;
    t.from_cache = 0;
    apply_tuning(net, t);
    if (cache_path && !cache_store(cache_path, key, t))
        return fail(VBMC_ERR_ARG, "autotune: cannot write the cache file");
    if (out) *out = t;
    return VBMC_OK;
}

extern "C" vbmc_status vbmc_fp8_accumulation_unit(vbmc_net* net, double* unit) {
    if (!net || !unit) return fail(VBMC_ERR_ARG, "null argument");
    if (!wide_supported(net->v))
        return fail(VBMC_ERR_UNSUPPORTED, "FP8 screen needs a ReLU net with hidden widths a multiple of 256 up to 1024");
    const vbmc_status st = wide_build(net->wide, net->v, net->hW, WIDE_E4M3);
    if (st != VBMC_OK) return fail(st, "FP8 set-up failed (self-test or weight preparation)");
    *unit = (double)net->wide.prec[WIDE_E4M3].acc_unit;
    return VBMC_OK;
}

extern "C" vbmc_status vbmc_net_prepare(vbmc_net* net, int32_t precision) {
    if (!net) return fail(VBMC_ERR_ARG, "null argument");
    if (precision < 0 || precision > VBMC_PREC_FP8) return fail(VBMC_ERR_ARG, "bad precision");
    if (precision == VBMC_PREC_FP64 || precision == VBMC_PREC_FP32) return VBMC_OK;
    const NetView& v = net->v;
    if ((precision == VBMC_PREC_BF16 || precision == VBMC_PREC_FP16) && tc_supported(v, precision)) {
        const vbmc_status st = tc_build(net->tc, v, net->hW, net->hb, precision);
        return st == VBMC_OK ? VBMC_OK : fail(st, "tensor-core set-up failed");
    }
    if (!wide_supported(v)) return fail(VBMC_ERR_UNSUPPORTED, "no tensor-core path for this net and precision");
    const vbmc_status st = wide_build(net->wide, v, net->hW, wide_type(precision));
    return st == VBMC_OK ? VBMC_OK : fail(st, "wide-layer tensor set-up failed (self-test or weight preparation)");
}

extern "C" vbmc_status vbmc_tc_accumulation_unit(vbmc_net* net, int32_t precision, double* unit, double* worst,
                                                  int32_t* probes_failed) {
    if (!net || !unit) return fail(VBMC_ERR_ARG, "null argument");
    if (precision != VBMC_PREC_BF16 && precision != VBMC_PREC_FP16)
        return fail(VBMC_ERR_ARG, "precision must be VBMC_PREC_BF16 or VBMC_PREC_FP16");
    float u = 0.f;
    double w = 0.0;
    int pf = 0;
    const vbmc_status st = tc_f16_selftest(precision == VBMC_PREC_BF16, &u, &w, &pf);
    if (st != VBMC_OK) return fail(st, "kind::f16 accumulator self-test failed or found no usable unit");
    *unit = (double)u;
    if (worst) *worst = w;
    if (probes_failed) *probes_failed = pf;
    return VBMC_OK;
}

extern "C" vbmc_status vbmc_shell_search(vbmc_net* net, const vbmc_query* q, const vbmc_options* opt,
                                         vbmc_result* res, vbmc_shell_out* out, void* stream) {
    if (!net || !q || !opt || !res) return fail(VBMC_ERR_ARG, "null argument");
    if (q->lo != 0 || q->hi != 0) return fail(VBMC_ERR_ARG, "a shell search covers whole shells: lo and hi must be 0");
    vbmc_shell_out so{-1, 0, 0, 0.0};
    for (int r = 0; r <= q->k; ++r) {
        vbmc_query qr = *q;
        qr.k = r;
        qr.filter = q->filter | VBMC_FILTER_SHELL;
        const vbmc_status st = vbmc_verify_query(net, &qr, opt, res, stream);
        if (st != VBMC_OK) return st;
        so.points_checked += res->sum.n_points;
        so.n_ties += res->sum.n_ties;
        so.ms_device += res->sum.ms_device;
        if (res->sum.n_adversarial > 0) {
            so.radius = r;
            break;
        }
    }
    if (out) *out = so;
    return VBMC_OK;
}
