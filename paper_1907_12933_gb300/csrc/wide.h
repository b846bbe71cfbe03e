// wide.h -- tensor-core screen for wide ReLU nets (hidden layers of 256..1024
// neurons), one layer per launch over chunks of points (internal).
#pragma once
#include "../../include/vbmc.h"
#include "dev.cuh"

#include <cudaTypedefs.h>
#include <vector>

namespace vbmc {

// Operand types of the wide path.
enum { WIDE_E4M3 = 0, WIDE_BF16 = 1, WIDE_FP16 = 2, WIDE_NTYPES = 3 };

constexpr int kWideFcap = 4;  // sign changes kept per point and layer (SS-Cover needs one)
constexpr int kWideOut = 32;  // classes (output width) the path supports
// Accumulation error per product of the tensor-core MMA, relative to sum
// |products|. The 16-bit kinds take the unit their set-up probe measures
// (tc_f16_selftest: 2^-22, the FP32 model, when exact). FP8 tensor-core
// accumulators have been reported to keep fewer bits than FP32 on earlier
// parts: the E4M3 set-up self-test adds probe sums whose exact values need 18
// to 23 significand bits, and the bound takes 2^-22 only when the MMA returns
// them exactly, 2^-13 otherwise.
constexpr float kWideAccFp32 = 0x1p-22f;
constexpr float kWideAccShort = 0x1p-13f;

// Hidden layer l >= 2 as a GEMM on rounded weights What = diag(sw) Wq (E4M3:
// sw_n = max_k |W_nk| / 448, Wq = e4m3(W / sw); 16-bit: sw = 1, Wq = round(W)).
struct WideLayer {
    int K = 0, N = 0;
    const void* wq = nullptr;     // [N][K]
    const float* sw = nullptr;    // [N] per-output-channel scale
    const float* a = nullptr;     // [N] ||What_n||_2 (rounded up)
    const float* b = nullptr;     // [N] ||W_n - What_n||_2 (rounded up)
    float sq = 0, sd = 0, fq = 0; // spectral bounds of What and W - What, ||What||_F
    CUtensorMap tw;               // Wq, box 128 bytes x 256 rows, 128-byte swizzle
};

struct WidePrec {
    bool ready = false;
    float acc_unit = kWideAccShort;
    WideLayer ly[kMaxL + 1];
};

struct WideNet {
    WidePrec prec[WIDE_NTYPES];
    std::vector<void*> owned;
};

// Per-result workspace of one chunk of points.
struct WideWork {
    unsigned long long chunk = 0;  // points per chunk
    int row_bytes = 0;             // bytes per operand row (2 x widest hidden layer)
    uint8_t* A[2] = {nullptr, nullptr};           // operand of layer l in A[l % 2]
    CUtensorMap tA[WIDE_NTYPES][2][kMaxL + 1];    // per operand type, buffer, layer
    // per layer l (1..L-1), per point: scale of the rounded operand of dh_l, sums
    // of squares of dh_l and of its rounding residual, and N, R, E of dh_l
    float* scale = nullptr;
    float* n2 = nullptr;
    float* r2 = nullptr;
    float* sN = nullptr;
    float* sR = nullptr;
    float* sE = nullptr;
    unsigned char* unc = nullptr;  // [chunk]: 1 some sign was not certain, 2 outside the filter
    int* fcnt = nullptr;           // [kMaxL + 1][chunk]: certain sign changes per layer
    short* flist = nullptr;        // [kMaxL + 1][chunk][kWideFcap]
    std::vector<void*> owned;
};

// The operand type of a precision, or -1.
int wide_type(int precision);
bool wide_supported(const NetView& v);
vbmc_status wide_build(WideNet& wn, const NetView& v, const std::vector<std::vector<float>>& W, int type);
void wide_free(WideNet& wn);
// Workspace for chunks of `chunk` points (0: the default 2^20), rounded up to 128.
vbmc_status wide_work_alloc(WideWork& w, const NetView& v, unsigned long long chunk);
void wide_work_free(WideWork& w);

// Diagnostic: while set, the first chunk of a wide-path run copies each hidden
// layer's operand rows (dequantized: the value times the point's scale) for its
// first n points into vals [(L-1)][n][hmax], and N, R, E of dh_l into nre
// [(L-1)][n][3] (device buffers).
struct WideTrace {
    float* vals = nullptr;
    float* nre = nullptr;
    int n = 0;
    int hmax = 0;
};
void wide_set_trace(const WideTrace* t);

// Screen [lo, hi) of query d_q[0] chunk by chunk. Each chunk's undecided points
// go through the FP32 (queue level 1), double-float (2) and FP64 (3) passes
// before the next chunk starts; the queue counters are reset per chunk.
vbmc_status wide_run(const WideNet& wn, int type, WideWork& w, const NetView& v, QueryView* d_q,
                     unsigned long long lo, unsigned long long hi, unsigned long long* d_qcount,
                     QEntry* const* d_queue, unsigned long long cap, int n_sm, cudaStream_t st);

}  // namespace vbmc
