// tc.h -- tensor-core (tcgen05) screen of layers 2..L (internal).
#pragma once
#include "../../include/vbmc.h"
#include "dev.cuh"

#include <cudaTypedefs.h>
#include <vector>

namespace vbmc {

constexpr int kTcMaxL = 6;     // weight layers the tensor path supports
constexpr int kTcMaxOut = 32;  // classes (output width) it supports

// Per layer l >= 2 of the tensor screen.
struct TcLayer {
    int K, N, Npad;        // inputs, outputs, outputs padded to the MMA width
    int slice, nslice;     // N per MMA / weight tile (<= 128) and slices per K chunk
    int kch;               // K / 64 chunks
    const float* a;        // [Npad] ||Wq_i||_2 (rounded up)
    const float* b1;       // [Npad] ||W_i - Wq_i||_2           (one-term screen)
    const float* b3;       // [Npad] ||W_i - Wq_i - Wlo_i||_2   (split screen)
    const void* wq;        // [Npad][K] 16-bit Wq (device), and Wlo
    const void* wlo;
    float sq, sa, sl;      // spectral-norm bounds of Wq, Wq + Wlo, Wlo
    float sd1, sd3;        // spectral-norm bounds of W - Wq, W - Wq - Wlo
    float fq;              // ||Wq||_F (1 + 2^-7) >= ||Wq + Wlo||_F
};

struct TcParams {
    CUtensorMap tq[kTcMaxL + 1];   // Wq_l  [Npad][K], box 64 x slice, 128-byte swizzle
    CUtensorMap tlo[kTcMaxL + 1];  // Wlo_l (split screen)
    TcLayer ly[kTcMaxL + 1];
    const float* pair;             // [H_L][H_L][5]: output-layer pair constants
    int L;
    int bf16;                      // 1: bf16 operands, 0: fp16
    float acc_unit;                // MMA accumulation error per product (tc_f16_selftest)
    int compact;                   // 1: per-query compacted columns (tq/tlo then map the
                                   // query's own weight copies; hidden layers in 128-row slices)
};

// Per-result workspace of the compacted screen: the query's copies of Wq_l and
// Wlo_l (l >= 2) with rows and columns in compacted order, and their tensor maps
// per operand type (encoded on first use; no allocation after creation).
struct TcQueryWork {
    void* wq[kTcMaxL + 1] = {};
    void* wlo[kTcMaxL + 1] = {};
    bool maps[2] = {false, false};  // [0] bf16, [1] fp16
    CUtensorMap tq[2][kTcMaxL + 1], tlo[2][kTcMaxL + 1];
    std::vector<void*> owned;
};

struct TcPrec {
    bool ready = false;
    TcParams p{};
};

struct TcNet {
    TcPrec prec[2];                // [0] bf16, [1] fp16
    // per-query class masks live in the result; see tc.cu
    std::vector<void*> owned;
};

bool tc_supported(const NetView& v, int precision);
// Measures the kind::f16 MMA accumulation unit on this device (see tc.cu):
// 2^-22 (the FP32 model) or 2^-13; VBMC_ERR_UNSUPPORTED when neither holds.
vbmc_status tc_f16_selftest(bool bf16, float* unit, double* worst, int* failed);
vbmc_status tc_build(TcNet& tc, const NetView& v, const std::vector<std::vector<float>>& W,
                     const std::vector<std::vector<float>>& b, int precision);
void tc_free(TcNet& tc);
// Allocates the compaction workspace of a result (the net's tensor path shapes).
vbmc_status tc_query_work_alloc(TcQueryWork& w, const NetView& v);
void tc_query_work_free(TcQueryWork& w);
// Per-query constants of the tensor screen (column classes), after the prologue;
// with qw (one query) also its compacted columns and weight copies.
void tc_launch_query_setup(TcNet& tc, const NetView& v, QueryView* d_q, int nq, int precision,
                           cudaStream_t st, TcQueryWork* qw = nullptr);
// Screen over nq queries: tiles of query q are d_tile_prefix[q] .. d_tile_prefix[q+1]-1
// (ntiles in total), each tc_tile_points() consecutive indices from (lo & ~31).
// qw: the compacted operands of the (single) query, prepared by the set-up.
// d_claim: the launch's tile claim counter (zeroed here; tiles are then taken in
// order under the queries' time budget, see claim_tile), or null for static tiles.
vbmc_status tc_launch_screen(TcNet& tc, const NetView& v, const QueryView* d_q, int nq,
                             const unsigned long long* d_tile_prefix, unsigned long long ntiles,
                             int precision, Queue out, int out_level, int n_sm, cudaStream_t st,
                             TcQueryWork* qw = nullptr, unsigned long long* d_claim = nullptr);
int tc_tile_points();
vbmc_status tc_launch_gather(TcNet& tc, const NetView& v, const QueryView* d_q, const QEntry* in,
                             const unsigned long long* in_count, unsigned long long cap,
                             int precision, Queue out, int n_sm, cudaStream_t st,
                             TcQueryWork* qw = nullptr);

}  // namespace vbmc
