// tc.cu -- tensor-core screen: layers 2..L of every point on tcgen05, BF16 or FP16
// operands, FP32 accumulation in TMEM, weights by TMA, error bound per point.
//
// CTA = 128 points (one MMA M). Warp roles:
//   warp 0      TMA producer: weight tiles [slice x 64] of W_l (K-major,
//               128-byte swizzle) into a ring of NB 16 KB slots
//   warp 1      TMEM owner (512 columns) and MMA issuer (one thread)
//   warps 2..17 workers: build the layer-2 operand (incremental layer 1,
//               Eq. 1, from the delta tables), drain each layer's
//               accumulator from TMEM, apply ReLU in delta form, quantise to
//               16-bit into the next layer's operand ring (NA 16 KB slots of
//               128 rows x 64 K), and finish each point: margin and class
//               (Eq. 10), sign changes and SS-Cover pairs (Sec. III-B).
//
// Delta form: every layer carries dh_l = h_l(point) - h_l(unperturbed image);
// the FP64 values of the unperturbed image come from the prologue, so the
// 16-bit rounding error scales with ||dh||, not ||h||.
//
// Error bound of du_l,i (per point, all norms 2-norms, u_acc = 2^-22 per
// accumulated product, Wq = rounded weights, Wr = W - Wq [- Wlo]):
//   |err| <= a_i (R + E + rho Lo + u_acc n (N + R + Lo)) + b_i (N + E)
// with n the number of operand columns that can be nonzero, i.e. not of the
// column class "neg" (zero at every point of the box: a product that is exactly
// zero adds nothing to the accumulator, so only the n others can carry rounding), a_i = ||Wq_i (+ Wlo_i)||, b_i = ||Wr_i||, N = ||dh_{l-1}||,
// R = ||dh_{l-1} - hi - lo|| (exact residual of the operand split),
// Lo = ||lo||, E = bound on the error of dh_{l-1}. The error vector of a
// whole layer propagates with spectral-norm bounds (sigma), the margin with
// the norms of row differences of the output layer. Split mode (three
// products hi*Wq + lo*Wq + hi*Wlo) is the tighter second pass.
#include "dev.cuh"
#include "launch.h"
#include "tc.h"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

namespace vbmc {

namespace {

constexpr int NW = 16;                   // worker warps
constexpr int NWT = 32 * NW;             // worker threads
constexpr int TC_THREADS = 64 + NWT;     // + TMA producer warp + MMA warp
constexpr int RPW = 128 / NW;            // layer-1 rows per worker warp
constexpr int CQ = NW / 4;               // worker warps per TMEM lane quarter
constexpr int CW = 64 / CQ;              // drain: columns of a 64-column chunk per warp
constexpr int kPfx0 = 160;               // decode phase: worker threads from here sum the prefixes
constexpr int NA = 4;
constexpr int NB = 4;
constexpr int kStageR = 16;  // layer-1 inner-digit tables are staged in shared memory for R <= kStageR
constexpr int kStageAll = 4; // with at most this many 64-column chunks, all of them at the tile's start
constexpr int SLOT = 16384;             // operand slot: 128 rows x 64 K (16-bit)
constexpr int SLOTB = 16384;             // weight slot: 128 rows (one N slice) x 64 K
constexpr int FCAP = 4;
constexpr int PMAX = 4;
constexpr int MROWS = 128;
// floats of the layer-1 staging union past the per-row input changes
constexpr int kWgen = kStageAll * 2 * kStageR * 64 - MROWS * kMaxS;

struct TcSmem {
    uint8_t A[NA][SLOT];
    uint8_t B[NB][SLOTB];
    float souter[PMAX][512];
    unsigned long long t[MROWS];
    int valid[MROWS];
    int pidx[MROWS];
    int4 rinfo[MROWS];     // layer-1 fast path: {prefix slot, inner table offsets a, b, valid}
    int4 winfo[NW];        // pair path: per worker warp {souter offset, digit s-2, digit s-1 of its
                           // first row, first row of the next (prefix, digit s-2) pair (RPW: none)}
    int2 winfo2[NW];       //   and that next pair's {souter offset, digit s-2}
    int fast;              // every valid row of the tile uses the fast path
    int pixs[kMaxS];       // the query's pixel indices
    float N[MROWS], R[MROWS], Lo[MROWS], E[MROWS];
    float nzl[kTcMaxL + 1];  // layer l: columns not in the class "neg" (the others are 0 at every point)
    float part[CQ][MROWS][3];
    int unc[MROWS];
    int vst[MROWS];
    int fcnt[MROWS][kTcMaxL + 1];
    short flist[MROWS][kTcMaxL + 1][FCAP];
    uint32_t cflip[256];   // sign changes seen by this CTA for query curq (flushed on change)
    // column constants of the layer in work, staged once per tile and layer from
    // the query's kcol arrays; thr' > 0 marks the class "cross" (ub', thr' are 0
    // for the other classes, whose signs are certain)
    float4 k1p[256];       // layer 1, per column pair (2i, 2i+1): (c1, c2, c1, c2)
    float4 k1u[256];       //   and (ub', thr', ub', thr') (read only where a column is "cross")
    uint2 k1cm[8];         //   per 64-column chunk: the "cross" columns 2 lane (x), 2 lane + 1 (y)
    float4 kd4[512];       // drained layer: (ub', ||Wq_i||, ||W_i - Wq_i (- Wlo_i)||, thr')
    float2 kd2[512];       //   and (c1, c2)
    union {
        // fast layer-1 path: tables of the two inner digits, one 64-column chunk, double-buffered
        float tstage[kStageAll][2][kStageR][64];
        // other tiles: per row and pixel fl(dv_p / 255), the pixel's input change
        float cpx[MROWS][kMaxS];
        // the same tiles: past cpx (from float MROWS * kMaxS on), the s weight rows
        // W_1[.][pix_p] of the layer-1 columns, when they fit
        float wgen[kStageAll * 2 * kStageR * 64];
    };
    int curq;
    int npref;
    unsigned long long claim[2];  // tile i of this CTA in claim[i & 1] (kNoTile: none left)
    int kch[kTcMaxL + 1];  // layer l: K chunks of 64 (compacted: the query's width of layer l-1)
    int nsl[kTcMaxL + 1];  //   N slices per K chunk
    int np[kTcMaxL + 1];   //   N computed (compacted: the query's width of layer l)
    int uniform_base;
    unsigned long long bars[2 * NB + 2 * NA + 7];
    uint32_t tmem_slot;
    int abort_flag;
};

static_assert(sizeof(TcSmem) + 1024 <= 227 * 1024, "tensor screen shared memory above the per-CTA limit");

// bar indices
__device__ __forceinline__ int BFULL(int i) { return i; }
__device__ __forceinline__ int BEMPTY(int i) { return NB + i; }
__device__ __forceinline__ int AFULL(int i) { return 2 * NB + i; }
__device__ __forceinline__ int AEMPTY(int i) { return 2 * NB + NA + i; }
// verdict flag bits of a point, ORed by the warps that share its outputs:
// Eq. 10: some margin pair certainly negative / some pair undecided;
// Eq. 11: y_D certainly above / below V, some other output certainly above V,
// some other output not certainly below V
enum : int {
    VF_UNSAFE = 1, VF_UNDECIDED = 2, VF_D_ABOVE = 4, VF_D_BELOW = 8, VF_O_ABOVE = 16, VF_O_NOT_BELOW = 32
};
constexpr int DFULL = 2 * NB + 2 * NA;
constexpr int TFREE = DFULL + 1;
constexpr int DRAINED = DFULL + 2;
constexpr int FIN = DFULL + 3;
__device__ __forceinline__ int CLAIMB(int i) { return DFULL + 4 + i; }  // claim[i] written

__device__ __forceinline__ float norm_up(float s) { return __fsqrt_ru(__fmul_ru(s, 1.0002f)); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Round two floats to a packed 16-bit pair (low half = first) and return the
// rounded values as floats.
template <bool BF>
__device__ __forceinline__ uint32_t pack2(float x, float y, float& qx, float& qy) {
    if (BF) {
        __nv_bfloat162 p = __floats2bfloat162_rn(x, y);
        qx = __low2float(p);
        qy = __high2float(p);
        return *reinterpret_cast<uint32_t*>(&p);
    } else {
        __half2 p = __floats2half2_rn(x, y);
        qx = __low2float(p);
        qy = __high2float(p);
        return *reinterpret_cast<uint32_t*>(&p);
    }
}

// Byte offset of 16-byte unit `u` (0..7) of row r in a 128-row x 128-byte slot,
// 128-byte swizzle (the layout TMA writes and the MMA descriptor reads).
__device__ __forceinline__ uint32_t sw_off(int r, int u) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((u ^ (r & 7)) << 4));
}

template <bool SPLIT, bool BF>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_tc(const __grid_constant__ TcParams P, NetView net, const QueryView* __restrict__ qs, int nq,
     const unsigned long long* __restrict__ tile_prefix, const QEntry* __restrict__ gather_in,
     const unsigned long long* __restrict__ gcount, unsigned long long gcap, Queue out,
     int out_level, unsigned long long* claim_ctr) {
    // the split pass always reads a queue (gather mode), the screen always ranges
    // (launch_k): the mode is known at compile time, and each instantiation keeps
    // only its own mode's code
    const QEntry* __restrict__ const gather = SPLIT ? gather_in : nullptr;
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned by pointer arithmetic on the shared array, so the compiler
    // keeps every access in the shared address space
    TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = P.L;
    volatile int* abortp = &S.abort_flag;

    // range mode: tiles of query q are tile_prefix[q] .. tile_prefix[q+1]-1, each
    // tile 128 consecutive indices from (lo & ~31); gather mode: 128 queue entries
    unsigned long long ntiles, gn = 0;
    if (SPLIT) {
        gn = *gcount;
        if (gn > gcap) gn = gcap;
        ntiles = (gn + MROWS - 1) / MROWS;
    } else {
        ntiles = tile_prefix[nq];
    }
    // range mode: tiles from the claim counter (in order, under the time budget);
    // gather mode: statically strided
    unsigned long long* const ctr = SPLIT ? nullptr : claim_ctr;
    const unsigned long long deadline =
        (!SPLIT && qs[0].budget_ns) ? qs[0].cnt->t0 + qs[0].budget_ns : 0ull;

    auto bar = [&](int i) { return tc::smem_u32(&S.bars[i]); };

    if (threadIdx.x == 0) {
        for (int i = 0; i < NB; ++i) {
            tc::mbar_init(bar(BFULL(i)), 1);
            tc::mbar_init(bar(BEMPTY(i)), 1);
        }
        for (int i = 0; i < NA; ++i) {
            tc::mbar_init(bar(AFULL(i)), NW);
            tc::mbar_init(bar(AEMPTY(i)), 1);
        }
        tc::mbar_init(bar(DFULL), 1);
        tc::mbar_init(bar(TFREE), NW);
        tc::mbar_init(bar(DRAINED), NW);
        tc::mbar_init(bar(FIN), 1);
        tc::mbar_init(bar(CLAIMB(0)), 1);
        tc::mbar_init(bar(CLAIMB(1)), 1);
        S.abort_flag = 0;
        S.curq = -1;
        S.claim[0] = claim_tile(ctr, 0, ntiles, deadline);  // this CTA's first tile
        // loop sizes per layer; compacted: the widths of the (single) query's
        // non-"neg" columns, rounded up to 64, from its set-up
        for (int l = 2; l <= L; ++l) {
            const TcLayer& ly = P.ly[l];
            const int Kc = P.compact ? qs[0].kc[l - 1] : ly.K;
            const int Nc = P.compact && l < L ? qs[0].kc[l] : ly.Npad;
            S.kch[l] = Kc / 64;
            S.np[l] = Nc;
            S.nsl[l] = (Nc + ly.slice - 1) / ly.slice;  // the last slice may be narrower
        }
        tc::fence_mbar_init();
    }
    for (int w = threadIdx.x; w < 256; w += blockDim.x) S.cflip[w] = 0u;
    if (warp == 1) {
        tc::tmem_alloc(tc::smem_u32(&S.tmem_slot), 512);
        tc::tmem_relinquish();
    }
    if (warp == 0 && lane == 0)
        for (int l = 2; l <= L; ++l) {
            tc::prefetch_tmap(&P.tq[l]);
            if (SPLIT) tc::prefetch_tmap(&P.tlo[l]);
        }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = S.tmem_slot;
    if (threadIdx.x == 0) tc::mbar_arrive(bar(CLAIMB(0)));  // claim[0] holds tile 0

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (uint32_t ti = 0; ok; ++ti) {
                if (!tc::mbar_wait(bar(CLAIMB(ti & 1)), (ti >> 1) & 1, abortp)) { ok = false; break; }
                if (S.claim[ti & 1] == kNoTile) break;
                for (int l = 2; l <= L && ok; ++l) {
                    const TcLayer& ly = P.ly[l];
                    for (int kc = 0; kc < S.kch[l] && ok; ++kc)
                        for (int s = 0; s < S.nsl[l] && ok; ++s)
                            for (int part = 0; part < (SPLIT ? 2 : 1); ++part) {
                                const int slot = it % NB;
                                if (!tc::mbar_wait(bar(BEMPTY(slot)), ((it / NB) & 1) ^ 1, abortp)) {
                                    ok = false;
                                    break;
                                }
                                tc::mbar_expect_tx(bar(BFULL(slot)), (uint32_t)ly.slice * 128u);
                                tc::tma_load_2d(tc::smem_u32(S.B[slot]), part ? &P.tlo[l] : &P.tq[l],
                                                kc * 64, s * ly.slice, bar(BFULL(slot)));
                                ++it;
                            }
                }
            }
            if (!ok) {  // let the copies already issued land before the CTA leaves
                const uint64_t t0 = tc::global_ns();
                for (uint32_t i = it > (uint32_t)NB ? it - NB : 0; i < it; ++i)
                    while (!tc::mbar_try(bar(BFULL(i % NB)), (i / NB) & 1) &&
                           tc::global_ns() - t0 < tc::kWaitNs) {
                    }
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            uint32_t ait = 0, bit = 0, tile_i = 0, drit = 0;
            bool ok = true;
            for (;; ++tile_i) {
                if (!tc::mbar_wait(bar(CLAIMB(tile_i & 1)), (tile_i >> 1) & 1, abortp)) { ok = false; break; }
                if (S.claim[tile_i & 1] == kNoTile) break;
                if (!tc::mbar_wait(bar(TFREE), (tile_i & 1) ^ 1, abortp)) { ok = false; break; }
                tc::tc_fence_after();
                for (int l = 2; l <= L && ok; ++l) {
                    const TcLayer& ly = P.ly[l];
                    if (l >= 3 && S.np[l] > 64) {
                        if (!tc::mbar_wait(bar(DRAINED), drit & 1, abortp)) { ok = false; break; }
                        ++drit;
                        tc::tc_fence_after();
                    }
                    // N of each slice: ly.slice, the last one what is left (a multiple of 64)
                    for (int kc = 0; kc < S.kch[l] && ok; ++kc) {
                        const int a0 = ait % NA, a1 = (ait + 1) % NA;
                        if (!tc::mbar_wait(bar(AFULL(a0)), (ait / NA) & 1, abortp)) { ok = false; break; }
                        if (SPLIT && !tc::mbar_wait(bar(AFULL(a1)), ((ait + 1) / NA) & 1, abortp)) {
                            ok = false;
                            break;
                        }
                        tc::tc_fence_after();
                        const uint32_t ab0 = tc::smem_u32(S.A[a0]), ab1 = tc::smem_u32(S.A[a1]);
                        for (int s = 0; s < S.nsl[l] && ok; ++s) {
                            const int b0 = bit % NB, b1 = (bit + 1) % NB;
                            if (!tc::mbar_wait(bar(BFULL(b0)), (bit / NB) & 1, abortp)) { ok = false; break; }
                            if (SPLIT && !tc::mbar_wait(bar(BFULL(b1)), ((bit + 1) / NB) & 1, abortp)) {
                                ok = false;
                                break;
                            }
                            tc::tc_fence_after();
                            const uint32_t bb0 = tc::smem_u32(S.B[b0]), bb1 = tc::smem_u32(S.B[b1]);
                            const uint32_t d = tmem + (uint32_t)(s * ly.slice);
                            const uint32_t idesc = tc::idesc_f16(128, min(ly.slice, S.np[l] - s * ly.slice), BF);
#pragma unroll
                            for (int ks = 0; ks < 4; ++ks) {
                                const uint64_t ad = tc::desc_sw128(ab0 + ks * 32);
                                const uint64_t bd = tc::desc_sw128(bb0 + ks * 32);
                                tc::mma_f16(d, ad, bd, idesc, (kc | ks) != 0);
                                if (SPLIT) {
                                    tc::mma_f16(d, tc::desc_sw128(ab1 + ks * 32), bd, idesc, 1);
                                    tc::mma_f16(d, ad, tc::desc_sw128(bb1 + ks * 32), idesc, 1);
                                }
                            }
                            tc::mma_commit(bar(BEMPTY(b0)));
                            if (SPLIT) tc::mma_commit(bar(BEMPTY(b1)));
                            bit += SPLIT ? 2 : 1;
                        }
                        tc::mma_commit(bar(AEMPTY(a0)));
                        if (SPLIT) tc::mma_commit(bar(AEMPTY(a1)));
                        ait += SPLIT ? 2 : 1;
                    }
                    tc::mma_commit(bar(DFULL));
                }
            }
            // everything issued must finish before TMEM is released
            tc::mma_commit(bar(FIN));
            const uint64_t t0 = tc::global_ns();
            while (!tc::mbar_try(bar(FIN), 0) && tc::global_ns() - t0 < tc::kWaitNs) {
            }
        }
    } else {
        // -------------------------------------------------------------- workers
        const int wid = warp - 2;            // 0..NW-1
        const int wtid = threadIdx.x - 64;   // 0..NWT-1
        const int qd = warp & 3;             // TMEM lane quarter
        const int hf = wid >> 2;             // column part (of CQ) in the drain phases
        const int H0 = net.dims[0], H1 = net.dims[1];
        uint32_t ait = 0, dit = 0;
        const float uacc_base = P.acc_unit * (SPLIT ? 3.f : 1.f);  // measured by tc_f16_selftest
        (void)H0;
        const bool cmp = P.compact != 0;  // compacted columns (one query): positions -> neurons by perm
        // The next tile's claim and the previous tile's count of finished work (time to
        // verdict) are global atomics: a worker thread without a row, a prefix sum or a
        // pixel in the decode issues them at the tile's start and publishes the claim at
        // the decode's end, so their latency overlaps the decode.
        constexpr int kAtomT = MROWS;
        static_assert(kAtomT < kPfx0 && kAtomT < MROWS + 64, "the atomics' thread has no decode row");
        Counters* pend_c = nullptr;    // thread kAtomT: the previous tile's finished units
        unsigned long long pend_n = 0;
        // the query whose staged column constants (layer 1; the drain of the one hidden
        // layer of a two-hidden-layer net) are in shared memory: restaged on a change
        int kq1 = -1, kqd = -1;
        for (uint32_t ti = 0;; ++ti) {
            if (*abortp) break;
            const unsigned long long g = S.claim[ti & 1];  // written before a barrier the workers passed
            if (g == kNoTile) break;
            unsigned long long nxt = kNoTile;
            if (wtid == kAtomT) {
                nxt = claim_tile(ctr, ti + 1, ntiles, deadline);
                if (pend_n) work_done(pend_c, pend_n);  // after the barrier that followed its pushes
                pend_n = 0;
            }
            int q = 0;
            if (!SPLIT) {
                int a = 0, b = nq - 1;
                while (a < b) {
                    const int mid = (a + b + 1) >> 1;
                    if (tile_prefix[mid] <= g) a = mid; else b = mid - 1;
                }
                q = a;
            }
            const QueryView& Q = qs[q];
            const int s = Q.s, R = Q.R;
            const int ni = s >= 2 ? 2 : s;       // inner digits handled per row
            unsigned long long Rni = 1;
            for (int i = 0; i < ni; ++i) Rni *= (unsigned long long)R;
            const unsigned long long base = Q.lo & ~31ull;
            const unsigned long long gq = SPLIT ? 0 : g - tile_prefix[q];
            if (q != S.curq) {  // this CTA's sign changes belong to the previous query
                const int cq = S.curq;
                if (cq >= 0)
                    for (int w = wtid; w < net.flip_words && w < 256; w += NWT)
                        if (S.cflip[w]) {
                            if (qs[cq].flip) atomicOr(&qs[cq].flip[w], S.cflip[w]);
                            S.cflip[w] = 0u;
                        }
                tc::named_bar_sync(1, NWT);
                if (wtid == 0) S.curq = q;
                if (wtid >= 1 && wtid < L) {  // operand entries that can be nonzero, per hidden layer
                    int c = 0;
                    for (int w = 0; w < (net.dims[wtid] + 31) / 32; ++w) c += __popc(~Q.cneg[wtid * 32 + w]);
                    S.nzl[wtid] = (float)min(c, net.dims[wtid]);
                }
                tc::named_bar_sync(1, NWT);
            }
            // ---- decode the tile's points. Range mode: the tile's indices are
            // consecutive, so their outer prefixes t / R^ni (the digits above the ni
            // inner ones) are consecutive integers from p0, that of the tile's first
            // index in [lo, hi): row r uses prefix slot t / R^ni - p0 when below PMAX.
            const bool pre = !SPLIT && s > ni;
            unsigned long long p0 = 0, np_need = 0;
            if (pre) {
                const unsigned long long t0 = base + gq * MROWS;
                const unsigned long long ta = t0 > Q.lo ? t0 : Q.lo;
                const unsigned long long tb = (t0 + MROWS < Q.hi ? t0 + MROWS : Q.hi) - 1;
                if (tb < 0xFFFFFFFFull && Rni < 0xFFFFFFFFull) {  // 32-bit division when it fits
                    p0 = (unsigned)ta / (unsigned)Rni;
                    np_need = (unsigned)tb / (unsigned)Rni - p0 + 1;
                } else {
                    p0 = ta / Rni;
                    np_need = tb / Rni - p0 + 1;
                }
            }
            const int np = (int)(np_need < (unsigned long long)PMAX ? np_need : PMAX);
            // fast layer-1 path: every valid row has its prefix slot (or s = 2: none needed);
            // with R <= kStageR its inner-digit tables come from shared memory
            const bool fast_t = !SPLIT && ((ni == 2 && s > 2 && np_need <= (unsigned long long)PMAX) || s == 2);
            const bool stage_t = fast_t && R <= kStageR;
            // layer-1 tables (compacted: column j' holds neuron perm_1[j']) and the
            // number of columns the dense layer 2 reads
            const float* __restrict__ tabq = cmp ? Q.tabc : Q.tab;
            const int W1cols = 64 * S.kch[2];
            if (stage_t && S.kch[2] <= kStageAll) {
                // the two inner digits' tables of every chunk, copied while the rows decode
                const int per = 2 * R * 16;  // 16-byte units per chunk
                for (int e = wtid; e < S.kch[2] * per; e += NWT) {
                    const int c = e / per, rem0 = e - c * per;
                    const int tt = rem0 / (R * 16), rem = rem0 - tt * (R * 16), dgt = rem >> 4, u = rem & 15;
                    cp_async16(&S.tstage[c][tt][dgt][4 * u],
                               tabq + ((size_t)(s - 2 + tt) * R + dgt) * H1 + 64 * c + 4 * u);
                }
                cp_async_commit();
            }
            if (wtid < MROWS) {
                const int r = wtid;
                unsigned long long t = 0;
                bool ok;
                if (SPLIT) {
                    const unsigned long long idx = g * MROWS + r;
                    ok = idx < gn;
                    if (ok) t = gather[idx].t;
                } else {
                    t = base + gq * MROWS + r;
                    ok = t >= Q.lo && t < Q.hi;
                }
                int d[kMaxS];
                const bool quick = fast_t && !Q.filter;  // only the two inner digits and the prefix
                unsigned long long tq = 0;               // t / R^ni (quick decode)
                if (quick) {
                    const unsigned long long tt = t;  // range mode: every row has its index
                    unsigned rr;
                    if (tt < 0xFFFFFFFFull && Rni < 0xFFFFFFFFull) {
                        const unsigned t32 = (unsigned)tt, r2 = (unsigned)Rni, q32 = t32 / r2;
                        tq = q32;
                        rr = t32 - q32 * r2;
                    } else {
                        tq = tt / Rni;
                        rr = (unsigned)(tt - tq * Rni);
                    }
                    d[s - 2] = (int)(rr / (unsigned)R);
                    d[s - 1] = (int)(rr - (unsigned)d[s - 2] * (unsigned)R);
                } else {
                    decode_digits(ok ? t : 0, s, R, d);
                }
                if (ok && !SPLIT && Q.filter) ok = in_filter(Q, d);  // L2 ball / shell
                if (!SPLIT && Q.filter) {  // points that pass the filter are counted here
                    const unsigned vm = __ballot_sync(0xffffffffu, ok);
                    if ((wtid & 31) == 0 && vm) atomicAdd(&Q.cnt->n_points, (unsigned long long)__popc(vm));
                }
                S.t[r] = t;
                S.valid[r] = ok;
                S.unc[r] = 0;
                S.vst[r] = 0;
#pragma unroll
                for (int l = 0; l <= kTcMaxL; ++l) S.fcnt[r][l] = 0;
                if (!fast_t)  // rows of the general layer-1 path: each pixel's input change
                    for (int p = 0; p < s; ++p) S.cpx[r][p] = __fdiv_rn((float)Q.dv[p * R + d[p]], 255.f);
                int pi = -1;
                if (pre && ok) {
                    const unsigned long long k = (quick ? tq : t / Rni) - p0;
                    if (k < (unsigned long long)PMAX) pi = (int)k;
                }
                S.pidx[r] = pi;
                // float offsets: the prefix slot's row of souter, and the rows of the two
                // inner-digit tables (staged chunk, or the global tables)
                int4 ri;
                ri.x = (pi >= 0 ? pi : 0) * 512;
                if (stage_t) {
                    ri.y = d[s - 2] * 64;
                    ri.z = (kStageR + d[s - 1]) * 64;
                } else {
                    ri.y = ni >= 2 ? ((s - 2) * R + d[s - 2]) * H1 : 0;
                    ri.z = ni >= 1 ? ((s - 1) * R + d[s - 1]) * H1 : 0;
                }
                ri.w = ok;
                S.rinfo[r] = ri;
                if (quick && stage_t && R >= RPW && (r % RPW) == 0) {
                    // the warp's RPW consecutive rows: digit s-1 runs up from its first row's
                    // and wraps at most once (R >= RPW), moving to the next (prefix, digit
                    // s-2) pair. Slots from the first row's true prefix offset (it may lie
                    // before lo: then every row of its pair does); rows outside [lo, hi)
                    // are masked off by their validity, so their slots are only clamped
                    const int d4 = d[s - 2], d5 = d[s - 1];
                    const int wrap = R - d5;  // first row of the next pair
                    const long long ka = pre ? (long long)tq - (long long)p0 : 0;
                    long long kb = ka;
                    int d4_b = d4 + 1;
                    if (d4_b == R) {
                        d4_b = 0;
                        kb = ka + 1;
                    }
                    const int sa = (int)(ka < 0 ? 0 : (ka >= PMAX ? PMAX - 1 : ka));
                    const int sb = (int)(kb < 0 ? 0 : (kb >= PMAX ? PMAX - 1 : kb));
                    S.winfo[r / RPW] = make_int4(sa * 512, d4, d5, wrap < RPW ? wrap : RPW);
                    S.winfo2[r / RPW] = make_int2(sb * 512, d4_b);
                }
            } else if (wtid >= MROWS + 64 && wtid - (MROWS + 64) < s) {
                S.pixs[wtid - (MROWS + 64)] = Q.pix[wtid - (MROWS + 64)];  // validated by the prologue
            }
            if (pre && wtid >= kPfx0) {
                // outer-prefix partial sums of layer 1, while the rows decode: slot k is
                // the prefix p0 + k (digits by carry from those of p0), summed over the
                // outer pixels in order
                int pd[kMaxS];
                decode_digits(p0, s - ni, R, pd);
                for (int k = 0; k < np; ++k) {
                    for (int j = wtid - kPfx0; j < W1cols; j += NWT - kPfx0) {
                        // unrolled so that the table loads are in flight together
                        // (the sum still runs over p in order)
                        float acc = 0.f;
#pragma unroll 4
                        for (int p = 0; p < s - ni; ++p) acc += __ldg(&tabq[((size_t)p * R + pd[p]) * H1 + j]);
                        S.souter[k][j] = acc;
                    }
                    for (int p = s - ni - 1; p >= 0; --p) {
                        if (++pd[p] < R) break;
                        pd[p] = 0;
                    }
                }
            }
            if (wtid == 0) {
                S.npref = np;
                S.fast = fast_t;
            }
            // general layer-1 path: the query's s weight rows, once per tile; the split
            // pass (one query, every tile on this path, nothing else in the region) once
            if (!fast_t && (!SPLIT || ti == 0)) {
                const int Wc = 64 * S.kch[2];
                if (s * Wc <= kWgen)
                    for (int e = wtid; e < s * Wc; e += NWT) {
                        const int p = e / Wc, jj = e - p * Wc;
                        S.wgen[MROWS * kMaxS + e] =
                            jj >= H1 ? 0.f : (cmp ? Q.w1c[(size_t)p * H1 + jj] : net.WT[1][(size_t)Q.pix[p] * H1 + jj]);
                    }
            }
            if (q != kq1) {  // the query's layer-1 column constants, for the build below: warp c
                // of the loop takes chunk c (its lanes the column pairs), whole warps only
                const float4* __restrict__ kcl = cmp ? Q.kcolc : Q.kcol;
                for (int e = wtid; e < 32 * S.kch[2]; e += NWT) {
                    const float4 kA0 = kcl[4 * e], kB0 = kcl[4 * e + 1];
                    const float4 kA1 = kcl[4 * e + 2], kB1 = kcl[4 * e + 3];
                    const bool cr0 = kB0.w == 2.f, cr1 = kB1.w == 2.f;
                    S.k1p[e] = make_float4(kB0.y, kB0.z, kB1.y, kB1.z);
                    S.k1u[e] = make_float4(cr0 ? kA0.x : 0.f, cr0 ? kB0.x : 0.f, cr1 ? kA1.x : 0.f, cr1 ? kB1.x : 0.f);
                    const unsigned m0 = __ballot_sync(0xffffffffu, cr0), m1 = __ballot_sync(0xffffffffu, cr1);
                    if ((e & 31) == 0) S.k1cm[e >> 5] = make_uint2(m0, m1);
                }
            }
            kq1 = q;
            if (wtid == kAtomT) {  // the producer and MMA warps learn the next tile
                S.claim[(ti + 1) & 1] = nxt;
                tc::mbar_arrive(bar(CLAIMB((ti + 1) & 1)));
            }
            cp_async_wait_all();  // this thread's table copies (staged at once) have landed
            tc::named_bar_sync(1, NWT);

            // ---- W1: layer-1 deltas -> operand of layer 2 (rows wid*RPW .. +RPW-1,
            //      lanes over column pairs 2*lane, 2*lane+1 of each 64-column chunk)
            {
                float nsum[RPW], rsum[RPW], lsum[RPW];
#pragma unroll
                for (int i = 0; i < RPW; ++i) nsum[i] = rsum[i] = lsum[i] = 0.f;
                const int kch = S.kch[2];
                const bool fast = S.fast;
                const bool nosum = (s == 2);  // fast path without outer digits
                // fast path with R <= kStageR: the tables of the two inner digits for a
                // chunk's 64 columns go to shared memory one chunk ahead (cp.async)
                const bool stage = fast && R <= kStageR;
                const bool pairs = stage && R >= RPW && !Q.filter;  // see winfo
                const unsigned wvalid = __ballot_sync(0xffffffffu, lane < RPW && S.valid[wid * RPW + lane]);
                auto stage_chunk = [&](int c, int buf) {
                    for (int e = wtid; e < 2 * R * 16; e += NWT) {
                        const int tt = e / (R * 16), rem = e - tt * (R * 16), dgt = rem >> 4, u = rem & 15;
                        cp_async16(&S.tstage[buf][tt][dgt][4 * u],
                                   tabq + ((size_t)(s - 2 + tt) * R + dgt) * H1 + 64 * c + 4 * u);
                    }
                    cp_async_commit();
                };
                // all chunks' tables were staged during the decode, or chunk by chunk here
                const bool stage_all = stage && kch <= kStageAll;
                if (stage && !stage_all) stage_chunk(0, 0);
                for (int c = 0; c < kch; ++c) {
                    const int a0 = ait % NA, a1 = (ait + 1) % NA;
                    tc::mbar_wait(bar(AEMPTY(a0)), ((ait / NA) & 1) ^ 1, abortp);
                    if (SPLIT) tc::mbar_wait(bar(AEMPTY(a1)), (((ait + 1) / NA) & 1) ^ 1, abortp);
                    const int sbuf = stage_all ? c : (c & 1);
                    if (stage && !stage_all) {
                        cp_async_wait_all();            // this thread's copies of chunk c
                        tc::named_bar_sync(1, NWT);     // everyone's; and chunk c-1's buffer is no longer read
                        if (c + 1 < kch) stage_chunk(c + 1, sbuf ^ 1);
                    }
                    const int j = 64 * c + 2 * lane;  // column (compacted: position) of this lane
                    // the columns' constants (staged for the tile, class folded in);
                    // dh = max(du + c1, c2) covers all classes: pos (0, -inf), neg (-inf, 0)
                    const float4 kp = S.k1p[32 * c + lane];
                    const uint2 cm = S.k1cm[c];
                    const bool cr0 = (cm.x >> lane) & 1u, cr1 = (cm.y >> lane) & 1u;
                    const bool anyc = (cm.x | cm.y) != 0u;  // warp-uniform
                    const float c10 = kp.x, c20 = kp.y, c11 = kp.z, c21 = kp.w;
                    float ub0 = 0.f, th0 = 0.f, ub1 = 0.f, th1 = 0.f;
                    if (anyc) {
                        const float4 ku = S.k1u[32 * c + lane];
                        ub0 = ku.x;
                        th0 = ku.y;
                        ub1 = ku.z;
                        th1 = ku.w;
                    }
                    const uint32_t lanepart = (lane & 3) * 4;
                    constexpr int RB = SPLIT ? (RPW < 4 ? RPW : 4) : (RPW < 8 ? RPW : 8);  // rows per batch
#pragma unroll
                    for (int i0 = 0; i0 < RPW; i0 += RB) {
                    // table sums of RB rows first (their loads overlap), then the rest
                    float2 dus[RB];
                    unsigned vbits = 0;  // valid rows of the batch (the compute loop stores to
                                         // shared memory, so it reloads nothing)
                    if (pairs) {
                        // the warp's rows share at most two (prefix, digit s-2) pairs: their
                        // sums souter + table(s-2) once per lane, then + table(s-1) per row,
                        // in the order of the per-row path
                        const int4 wa = S.winfo[wid];
                        const float* ts = &S.tstage[sbuf][0][0][2 * lane];
                        float2 s1a = nosum ? make_float2(0.f, 0.f)
                                           : *reinterpret_cast<const float2*>(&S.souter[0][0] + wa.x + j);
                        const float2 taa = *reinterpret_cast<const float2*>(ts + wa.y * 64);
                        s1a.x = s1a.x + taa.x;
                        s1a.y = s1a.y + taa.y;
                        float2 s1b = s1a;
                        if (wa.w < RPW) {  // warp-uniform
                            const int2 wb = S.winfo2[wid];
                            s1b = nosum ? make_float2(0.f, 0.f)
                                        : *reinterpret_cast<const float2*>(&S.souter[0][0] + wb.x + j);
                            const float2 tab_ = *reinterpret_cast<const float2*>(ts + wb.y * 64);
                            s1b.x = s1b.x + tab_.x;
                            s1b.y = s1b.y + tab_.y;
                        }
                        vbits = (wvalid >> i0) & ((1u << RB) - 1u);
#pragma unroll
                        for (int ii = 0; ii < RB; ++ii) {
                            const int i = i0 + ii;
                            const bool second = i >= wa.w;
                            const int d5 = wa.z + i - (second ? R : 0);
                            const float2 tb = *reinterpret_cast<const float2*>(ts + (kStageR + d5) * 64);
                            const float2 s1 = second ? s1b : s1a;
                            dus[ii] = make_float2(s1.x + tb.x, s1.y + tb.y);
                        }
                    } else if (fast) {
#pragma unroll
                        for (int ii = 0; ii < RB; ++ii) {
                            const int r = wid * RPW + i0 + ii;
                            const int4 ri = S.rinfo[r];
                            if (ri.w) vbits |= 1u << ii;
                            float2 du = nosum ? make_float2(0.f, 0.f)
                                              : *reinterpret_cast<const float2*>(&S.souter[0][0] + ri.x + j);
                            float2 ta, tb;
                            if (stage) {
                                const float* ts = &S.tstage[sbuf][0][0][2 * lane];
                                ta = *reinterpret_cast<const float2*>(ts + ri.y);
                                tb = *reinterpret_cast<const float2*>(ts + ri.z);
                            } else {
                                ta = __ldg(reinterpret_cast<const float2*>(&tabq[ri.y + j]));
                                tb = __ldg(reinterpret_cast<const float2*>(&tabq[ri.z + j]));
                            }
                            du.x = (du.x + ta.x) + tb.x;
                            du.y = (du.y + ta.y) + tb.y;
                            dus[ii] = du;
                        }
                    } else {
                        // general path: a row's outer-prefix sum when it has a slot, then
                        // W_1[j][pix_p] * fl(dv_p / 255) for its remaining pixels in order,
                        // each term fused into the sum (paired FMA over the lane's two
                        // columns: one rounding per term, against two in a table entry
                        // plus the sum, so inside the prologue's table-sum bound e1).
                        // The weight pair of pixel p is the same for every row: one load
                        // per pixel serves the batch.
                        int pfrom[RB];
#pragma unroll
                        for (int ii = 0; ii < RB; ++ii) {
                            const int r = wid * RPW + i0 + ii;
                            const int4 ri = S.rinfo[r];
                            if (ri.w) vbits |= 1u << ii;
                            const int pi = S.pidx[r];
                            dus[ii] = (ri.w && pi >= 0) ? *reinterpret_cast<const float2*>(&S.souter[pi][j])
                                                        : make_float2(0.f, 0.f);
                            pfrom[ii] = !ri.w ? s : (pi >= 0 ? s - ni : 0);
                        }
                        const int Wc = 64 * kch;
                        const bool wsh = s * Wc <= kWgen;  // the weight rows were staged (tile-uniform)
                        for (int p = 0; p < s; ++p) {
                            const float2 w2 = wsh ? *reinterpret_cast<const float2*>(&S.wgen[MROWS * kMaxS + p * Wc + j])
                                                  : __ldg(reinterpret_cast<const float2*>(
                                                        cmp ? &Q.w1c[(size_t)p * H1 + j] : &net.WT[1][(size_t)S.pixs[p] * H1 + j]));
#pragma unroll
                            for (int ii = 0; ii < RB; ++ii) {
                                if (p < pfrom[ii]) continue;
                                const float c = S.cpx[wid * RPW + i0 + ii][p];
                                dus[ii] = __ffma2_rn(w2, make_float2(c, c), dus[ii]);
                            }
                        }
                    }
#pragma unroll
                    for (int ii = 0; ii < RB; ++ii) {
                        const int i = i0 + ii;
                        const int r = wid * RPW + i;
                        const bool rw = (vbits >> ii) & 1u;
                        const float2 du = dus[ii];
                        float dh0 = fmaxf(du.x + c10, c20);
                        float dh1 = fmaxf(du.y + c11, c21);
                        if (!rw) dh0 = dh1 = 0.f;
                        if (anyc && rw && Q.flip) {  // signs matter only for coverage
                            if (cr0) {
                                const float u = ub0 + du.x;
                                if (!(__fmul_rd(fabsf(u), 1.f - 0x1p-22f) > th0)) S.unc[r] = 1;
                                else if ((u >= 0.f) != (ub0 >= 0.f)) {
                                    const int k = atomicAdd(&S.fcnt[r][1], 1);
                                    const int jo0 = cmp ? Q.perm[j] : j;  // the neuron
                                    if (k < FCAP) S.flist[r][1][k] = (short)jo0;
                                    atomicOr(&S.cflip[jo0 >> 5], 1u << (jo0 & 31));
                                }
                            }
                            if (cr1) {
                                const float u = ub1 + du.y;
                                if (!(__fmul_rd(fabsf(u), 1.f - 0x1p-22f) > th1)) S.unc[r] = 1;
                                else if ((u >= 0.f) != (ub1 >= 0.f)) {
                                    const int k = atomicAdd(&S.fcnt[r][1], 1);
                                    const int jo1 = cmp ? Q.perm[j + 1] : j + 1;  // the neuron
                                    if (k < FCAP) S.flist[r][1][k] = (short)jo1;
                                    atomicOr(&S.cflip[jo1 >> 5], 1u << (jo1 & 31));
                                }
                            }
                        }
                        float q0, q1;
                        const uint32_t w = pack2<BF>(dh0, dh1, q0, q1);
                        float r0 = dh0 - q0, r1 = dh1 - q1;
                        // r & 7 == i & 7 (wid * RPW is a multiple of 8): swizzle known per i
                        static_assert(RPW % 8 == 0, "rows of a warp start at a swizzle atom");
                        const uint32_t off = (uint32_t)((wid * (RPW / 8) + (i >> 3)) * 1024 + (i & 7) * 128) +
                                             ((((uint32_t)lane >> 2) ^ (uint32_t)(i & 7)) << 4) + lanepart;
                        *reinterpret_cast<uint32_t*>(&S.A[a0][off]) = w;
                        if (SPLIT) {
                            float l0, l1;
                            const uint32_t wl = pack2<BF>(r0, r1, l0, l1);
                            *reinterpret_cast<uint32_t*>(&S.A[a1][off]) = wl;
                            lsum[i] = fmaf(l0, l0, fmaf(l1, l1, lsum[i]));
                            r0 -= l0;
                            r1 -= l1;
                        }
                        nsum[i] = fmaf(dh0, dh0, fmaf(dh1, dh1, nsum[i]));
                        rsum[i] = fmaf(r0, r0, fmaf(r1, r1, rsum[i]));
                    }
                    }  // i0
                    tc::fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) {
                        tc::mbar_arrive(bar(AFULL(a0)));
                        if (SPLIT) tc::mbar_arrive(bar(AFULL(a1)));
                    }
                    ait += SPLIT ? 2 : 1;
                }
                // row sums over the warp (every lane ends with the totals), then lane i
                // bounds row i's norms: the square roots run in parallel over the lanes
                float tn = 0.f, tr = 0.f, tl = 0.f;
#pragma unroll
                for (int i = 0; i < RPW; ++i) {
                    float a = nsum[i], b = rsum[i], cc = lsum[i];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        a += __shfl_xor_sync(0xffffffffu, a, o);
                        b += __shfl_xor_sync(0xffffffffu, b, o);
                        if (SPLIT) cc += __shfl_xor_sync(0xffffffffu, cc, o);
                    }
                    if (lane == i) {
                        tn = a;
                        tr = b;
                        tl = cc;
                    }
                }
                if (lane < RPW) {
                    const int r = wid * RPW + lane;
                    const float N = norm_up(tn);
                    S.N[r] = N;
                    S.R[r] = norm_up(tr);
                    S.Lo[r] = SPLIT ? norm_up(tl) : 0.f;
                    S.E[r] = __fmaf_ru(0x1p-24f, N, Q.kvec[1]);
                }
            }
            tc::named_bar_sync(1, NWT);

            // ---- hidden layers: drain D_l, write the operand of layer l+1
            const int r = 32 * qd + lane;
            for (int l = 2; l < L; ++l) {
                const TcLayer& ly = P.ly[l];
                if (L > 3 || q != kqd) {  // this layer's column constants (the previous readers
                    // passed a barrier); their loads overlap the wait for the layer's MMAs
                    const float4* __restrict__ kcl = (cmp ? Q.kcolc : Q.kcol) + 2 * net.noff[l];
                    for (int e = wtid; e < S.np[l]; e += NWT) {
                        const float4 kA = kcl[2 * e], kB = kcl[2 * e + 1];
                        const bool cr = kB.w == 2.f;
                        S.kd4[e] = cr ? make_float4(kA.x, kA.y, SPLIT ? kA.w : kA.z, kB.x)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
                        S.kd2[e] = make_float2(kB.y, kB.z);
                    }
                }
                kqd = q;
                tc::mbar_wait(bar(DFULL), dit & 1, abortp);
                ++dit;
                tc::tc_fence_after();
                tc::named_bar_sync(1, NWT);  // the staged constants are visible
                const float Nn = S.N[r], Rr = S.R[r], Ll = S.Lo[r], Ee = S.E[r];
                // accumulation: 2^-22 per product that can be nonzero (an exact zero adds nothing)
                const float uacc = uacc_base * fminf(S.nzl[l - 1], (float)ly.K);
                const float Pa = __fmaf_ru(uacc, __fadd_ru(__fadd_ru(Nn, Rr), __fmul_ru(2.f, Ll)),
                                           __fmaf_ru(SPLIT ? 0x1p-7f : 0.f, Ll, __fadd_ru(Rr, Ee)));
                const float Pb = __fadd_ru(Nn, Ee);
                const int off_l = net.noff[l];
                float ns = 0.f, rs = 0.f, ls = 0.f;
                const int nch = S.np[l] / 64;
                for (int c = 0; c < nch; ++c) {
                    const int a0 = ait % NA, a1 = (ait + 1) % NA;
                    tc::mbar_wait(bar(AEMPTY(a0)), ((ait / NA) & 1) ^ 1, abortp);
                    if (SPLIT) tc::mbar_wait(bar(AEMPTY(a1)), (((ait + 1) / NA) & 1) ^ 1, abortp);
                    const int n0 = 64 * c + CW * hf;
                    float v[CW];
                    tc::tmem_ld<CW>(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)n0, v);
                    // the class of each of the warp's CW columns (lane i < CW: column n0 + i);
                    // compacted: position nl holds neuron perm_l[nl], positions past the
                    // count are "neg"
                    const bool cl = lane < CW;
                    const int nl = n0 + (cl ? lane : 0);
                    // the class "cross" of the warp's columns (thr' > 0; staged constants)
                    const uint32_t cross = __ballot_sync(0xffffffffu, cl && S.kd4[nl].w > 0.f);
                    const bool rv = S.valid[r];
                    if (cross && rv && Q.flip != nullptr) {  // signs matter only for coverage
                        // no stores in the loop (its loads pipeline): uncertain signs and
                        // certain changes as bits, handled after
                        // branch-free within groups of 8 columns (constants of the other
                        // classes are zero); the column class selects the bits afterwards
                        uint32_t uncb = 0u, flb = 0u;
#pragma unroll
                        for (int g = 0; g < CW / 8; ++g) {
                            if ((cross >> (8 * g)) & 0xFFu) {
#pragma unroll
                                for (int i = 8 * g; i < 8 * g + 8; ++i) {
                                    const float4 k4 = S.kd4[n0 + i];
                                    const float u = k4.x + v[i];
                                    const float bound = __fmaf_ru(k4.y, Pa, __fmaf_ru(k4.z, Pb, k4.w));
                                    const bool cert = __fmul_rd(fabsf(u), 1.f - 0x1p-22f) > bound;
                                    uncb |= (uint32_t)!cert << i;
                                    flb |= (uint32_t)(cert && ((u >= 0.f) != (k4.x >= 0.f))) << i;
                                }
                            }
                        }
                        uncb &= cross;
                        flb &= cross;
                        if (uncb) S.unc[r] = 1;
                        while (flb) {
                            const int nc = n0 + __ffs(flb) - 1;
                            const int n = cmp ? Q.perm[off_l + nc] : nc, gi = off_l + n;
                            flb &= flb - 1u;
                            const int k = atomicAdd(&S.fcnt[r][l], 1);
                            if (k < FCAP) S.flist[r][l][k] = (short)n;
                            atomicOr(&S.cflip[gi >> 5], 1u << (gi & 31));
                        }
                    }
                    // delta ReLU; no stores in this loop, so its loads pipeline
#pragma unroll
                    for (int i = 0; i < CW; ++i) {
                        const float2 k2 = S.kd2[n0 + i];
                        v[i] = fmaxf(v[i] + k2.x, k2.y);
                    }
                    __syncwarp();  // the staged constants are read before the next chunk overwrites them
                    if (!__all_sync(0xffffffffu, rv) && !rv) {
#pragma unroll
                        for (int i = 0; i < CW; ++i) v[i] = 0.f;
                    }
                    uint32_t wq[CW / 2], wl[CW / 2];
#pragma unroll
                    for (int i = 0; i < CW / 2; ++i) {
                        float q0, q1;
                        wq[i] = pack2<BF>(v[2 * i], v[2 * i + 1], q0, q1);
                        float r0 = v[2 * i] - q0, r1 = v[2 * i + 1] - q1;
                        if (SPLIT) {
                            float l0, l1;
                            wl[i] = pack2<BF>(r0, r1, l0, l1);
                            ls = fmaf(l0, l0, fmaf(l1, l1, ls));
                            r0 -= l0;
                            r1 -= l1;
                        }
                        ns = fmaf(v[2 * i], v[2 * i], fmaf(v[2 * i + 1], v[2 * i + 1], ns));
                        rs = fmaf(r0, r0, fmaf(r1, r1, rs));
                    }
#pragma unroll
                    for (int k = 0; k < CW / 8; ++k) {  // 16-byte units of the row's CW columns
                        const uint32_t o = sw_off(r, hf * (CW / 8) + k);
                        *reinterpret_cast<uint4*>(&S.A[a0][o]) =
                            make_uint4(wq[4 * k], wq[4 * k + 1], wq[4 * k + 2], wq[4 * k + 3]);
                        if (SPLIT)
                            *reinterpret_cast<uint4*>(&S.A[a1][o]) =
                                make_uint4(wl[4 * k], wl[4 * k + 1], wl[4 * k + 2], wl[4 * k + 3]);
                    }
                    tc::fence_proxy_async();
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        tc::mbar_arrive(bar(AFULL(a0)));
                        if (SPLIT) tc::mbar_arrive(bar(AFULL(a1)));
                    }
                    ait += SPLIT ? 2 : 1;
                }
                S.part[hf][r][0] = ns;
                S.part[hf][r][1] = rs;
                S.part[hf][r][2] = ls;
                tc::tc_fence_before();
                tc::named_bar_sync(1, NWT);
                if (hf == 0) {
                    float n2 = 0.f, r2 = 0.f, l2 = 0.f;
#pragma unroll
                    for (int h = 0; h < CQ; ++h) {
                        n2 += S.part[h][r][0];
                        r2 += S.part[h][r][1];
                        l2 += S.part[h][r][2];
                    }
                    const float N = norm_up(n2);
                    const float Rn = norm_up(r2);
                    const float Lo = norm_up(l2);
                    // ||err(du_l)|| <= sA R + sB N + (sA + sB) E + sL Lo + uacc fq (N + R + 2 Lo)
                    const float sA = SPLIT ? ly.sa : ly.sq, sB = SPLIT ? ly.sd3 : ly.sd1;
                    float El = __fmul_ru(sA, Rr);
                    El = __fmaf_ru(sB, Nn, El);
                    El = __fmaf_ru(__fadd_ru(sA, sB), Ee, El);
                    if (SPLIT) El = __fmaf_ru(ly.sl, Ll, El);
                    El = __fmaf_ru(__fmul_ru(uacc, ly.fq), __fadd_ru(__fadd_ru(Nn, Rr), __fmul_ru(2.f, Ll)), El);
                    El = __fadd_ru(El, Q.kvec[l]);
                    El = __fmaf_ru(0x1p-24f, N, El);
                    S.N[r] = N;
                    S.R[r] = Rn;
                    S.Lo[r] = Lo;
                    S.E[r] = El;
                }
                if (l + 1 < L && S.np[l + 1] > 64) {
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(bar(DRAINED));
                }
                tc::named_bar_sync(1, NWT);
            }

            // ---- output layer: margin (Eq. 10) or threshold literal (Eq. 11), output signs
            {
                const TcLayer& ly = P.ly[L];
                tc::mbar_wait(bar(DFULL), dit & 1, abortp);
                ++dit;
                tc::tc_fence_after();
                // the CQ warps of a TMEM lane quarter share the outputs: warp hf takes
                // outputs o = hf, hf + CQ, ...; their verdict parts meet in S.vst[r]
                // as flag bits (see VF_* below)
                {
                    float v[32];
                    tc::tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16), v);
                    if (S.valid[r]) {
                        const float Nn = S.N[r], Rr = S.R[r], Ll = S.Lo[r], Ee = S.E[r];
                        const float uacc = uacc_base * fminf(S.nzl[L - 1], (float)ly.K);
                        const float Pa = __fmaf_ru(uacc, __fadd_ru(__fadd_ru(Nn, Rr), __fmul_ru(2.f, Ll)),
                                                   __fmaf_ru(SPLIT ? 0x1p-7f : 0.f, Ll, __fadd_ru(Rr, Ee)));
                        const float Pb = __fadd_ru(Nn, Ee);
                        const float* av = ly.a;
                        const float* bv = SPLIT ? ly.b3 : ly.b1;
                        const int HL = ly.N, offL = net.noff[L];
                        const int D = Q.cnt->D;
                        float vD = 0.f;  // v[D] by selection (v stays in registers)
#pragma unroll
                        for (int o = 0; o < kTcMaxOut; ++o)
                            if (o == D) vD = v[o];
                        const float yD = Q.ub32[offL + D] + vD;
                        const float dD = Q.dub[offL + D];
                        const float* pr = P.pair + (size_t)D * HL * 5;
                        const bool thr = Q.prop == PROP_THRESHOLD;
                        bool unc = false;
                        int f = 0;
#pragma unroll
                        for (int o0 = 0; o0 < kTcMaxOut; o0 += CQ) {
                            const int o = o0 + hf;
                            if (o >= HL) break;
                            float vo = 0.f;  // v[o] by selection (v stays in registers)
#pragma unroll
                            for (int h = 0; h < CQ; ++h)
                                if (h == hf && o0 + h < kTcMaxOut) vo = v[o0 + h];
                            const float ub = Q.ub32[offL + o];
                            const float u = ub + vo;
                            const float bound = __fmaf_ru(av[o], Pa, __fmaf_ru(bv[o], Pb, Q.thr[offL + o]));
                            if (!(__fmul_rd(fabsf(u), 1.f - 0x1p-22f) > bound)) unc = Q.flip != nullptr;
                            else if ((u >= 0.f) != (ub >= 0.f)) {
                                const int k = atomicAdd(&S.fcnt[r][L], 1);
                                if (k < FCAP) S.flist[r][L][k] = (short)o;
                                atomicOr(&S.cflip[(offL + o) >> 5], 1u << ((offL + o) & 31));
                            }
                            if (thr) {  // Eq. 11: per output a_o Pa + b_o Pb + dub_o
                                const float e = __fmaf_ru(av[o], Pa, __fmaf_ru(bv[o], Pb, __fadd_ru(Q.dub[offL + o],
                                                                                              (float)(2.0 * kTau))));
                                const int sd = thr_side(u, (float)Q.V, e);
                                if (o == D) f |= (sd > 0 ? VF_D_ABOVE : 0) | (sd < 0 ? VF_D_BELOW : 0);
                                else f |= (sd > 0 ? VF_O_ABOVE : 0) | (sd < 0 ? 0 : VF_O_NOT_BELOW);
                            } else if (o != D) {  // Eq. 10: margin pair (D, o)
                                const float diff = yD - u;
                                const float* c5 = pr + o * 5;
                                float eb = __fmul_ru(c5[0], __fadd_ru(Rr, 0.f));
                                eb = __fmaf_ru(c5[1], Nn, eb);
                                eb = __fmaf_ru(c5[2], Ee, eb);
                                if (SPLIT) eb = __fmaf_ru(c5[3], Ll, eb);
                                eb = __fmaf_ru(__fmul_ru(uacc, c5[4]), __fadd_ru(__fadd_ru(Nn, Rr), __fmul_ru(2.f, Ll)), eb);
                                eb = __fadd_ru(eb, __fadd_ru(__fadd_ru(dD, Q.dub[offL + o]), (float)(2.0 * kTau)));
                                eb = __fmaf_ru(0x1p-23f, __fadd_ru(__fadd_ru(fabsf(yD), fabsf(u)), fabsf(diff)), eb);
                                if (diff < -eb) f |= VF_UNSAFE;
                                else if (!(diff > eb)) f |= VF_UNDECIDED;
                            }
                        }
                        if (f) atomicOr(&S.vst[r], f);
                        if (unc) S.unc[r] = 1;
                    }
                }
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(bar(TFREE));
                tc::named_bar_sync(1, NWT);
                // ---- per-point results: the warps of a lane quarter split the three
                // independent parts (queue, verdict counts and bitmap, SS-Cover bits)
                static_assert(CQ >= 3, "the results need three warps per lane quarter");
                if (hf < 3) {
                    const bool rv = S.valid[r];
                    const int vf = S.vst[r];
                    const int vv = Q.prop == PROP_THRESHOLD
                                       ? thr_verdict(vf & VF_D_ABOVE, vf & VF_D_BELOW, vf & VF_O_ABOVE,
                                                     !(vf & VF_O_NOT_BELOW))
                                       : ((vf & VF_UNSAFE) ? 1 : ((vf & VF_UNDECIDED) ? 2 : 0));
                    bool bad = rv && (S.unc[r] || vv == 2);
                    if (rv && !bad && Q.ss)
                        for (int l = 1; l < L; ++l)
                            if (S.fcnt[r][l] == 1 && S.fcnt[r][l + 1] > FCAP) bad = true;
                    const unsigned long long t = S.t[r];
                    const bool adv = rv && !bad && vv == 1;
                    if (hf == 0) {
                        queue_push_warp(out, bad, t, (unsigned)q, Q.cnt, out_level);
                    } else if (hf == 1 && !SPLIT) {
                        const unsigned m = __ballot_sync(0xffffffffu, adv);
                        if (m && lane == 0) {
                            atomicAdd(&Q.cnt->n_adv, (unsigned long long)__popc(m));
                            atomicMin(&Q.cnt->first, t + (unsigned)(__ffs(m) - 1));
                            if (Q.bitmap && t < Q.bitmap_bits) atomicOr(&Q.bitmap[t >> 5], m);
                        }
                    } else if (hf == 1 && adv) {
                        record_adversarial(Q, t);
                    } else if (hf == 2 && rv && !bad && Q.ss) {
                        for (int l = 1; l < L; ++l) {
                            if (S.fcnt[r][l] != 1) continue;  // SS needs exactly one change
                            const int j = S.flist[r][l][0];
                            const int Hn = net.dims[l + 1];
                            const int nt = S.fcnt[r][l + 1];
                            for (int e = 0; e < nt; ++e)
                                set_bit_once(Q.ss, (unsigned long long)net.ssoff[l] +
                                                       (unsigned long long)j * Hn + S.flist[r][l + 1][e]);
                        }
                    }
                }
                tc::named_bar_sync(1, NWT);
                // time to verdict: a screen tile done, or this tile's queued points resolved
                if (wtid == kAtomT) {  // counted at the next tile's start (or below)
                    pend_c = Q.cnt;
                    pend_n = SPLIT ? (g * MROWS + MROWS <= gn ? MROWS : gn - g * MROWS) : 1;
                }
            }
        }
        if (wtid == kAtomT && pend_n) work_done(pend_c, pend_n);
    }
    // ---- teardown: wait for outstanding tensor-core work, release TMEM
    tc::tc_fence_before();
    __syncthreads();
    if (S.curq >= 0 && qs[S.curq].flip)
        for (int w = threadIdx.x; w < net.flip_words && w < 256; w += blockDim.x)
            if (S.cflip[w]) atomicOr(&qs[S.curq].flip[w], S.cflip[w]);
    if (warp == 1) {
        __syncwarp();
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
    if (threadIdx.x == 0 && *abortp) atomicOr(&qs[S.curq >= 0 ? S.curq : 0].cnt->err, DERR_TC_WAIT);
}

// ------------------------------------------------------------ per-query setup

// Column classes of the tensor screen. A neuron whose |ub| exceeds a bound on
// |du| over the whole box plus the screen's error bound keeps its sign at every
// point: "pos" (output change = input change) or "neg" (output change 0). The
// bound on |du| propagates interval bounds |dh_j| <= B_j through |W_l|.
__global__ void k_classes_tc(const __grid_constant__ TcParams P, NetView net, QueryView* qs) {
    __shared__ double Bh[1024];
    __shared__ double red[64];
    QueryView& Q = qs[blockIdx.x];
    const int L = P.L, H1 = net.dims[1];
    const double u24 = 0x1p-24;
    const double uq = P.bf16 ? 0x1p-8 : 0x1p-11;
    // layer 1
    double part = 0.0;
    for (int w = threadIdx.x; w < (kMaxL + 1) * 32; w += blockDim.x) {
        Q.cpos[w] = 0u;
        Q.cneg[w] = 0u;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < H1; j += blockDim.x) {
        double b1 = 0.0;
        for (int p = 0; p < Q.s; ++p) {
            double mx = 0.0;
            for (int d = 0; d < Q.R; ++d)
                mx = fmax(mx, fabs((double)Q.tab[((size_t)p * Q.R + d) * H1 + j]));
            b1 += mx;
        }
        b1 *= 1.0 + 1e-6;
        const double ub = Q.ub[j];
        const bool cross = !(fabs(ub) > (b1 + (double)Q.thr[j]) * (1.0 + 1e-6) + 4.0 * kTau);
        if (!cross) atomicOr(ub >= 0.0 ? &Q.cpos[32 + (j >> 5)] : &Q.cneg[32 + (j >> 5)], 1u << (j & 31));
        Bh[j] = (!cross && ub < 0.0) ? 0.0 : b1;
        if (Q.kcol) {
            const int cls = cross ? 2 : (ub >= 0.0 ? 0 : 1);
            Q.kcol[2 * j] = make_float4(Q.ub32[j], 0.f, 0.f, 0.f);
            Q.kcol[2 * j + 1] = make_float4(Q.thr[j], cls == 2 ? Q.c1[j] : (cls == 0 ? 0.f : -INFINITY),
                                            cls == 2 ? Q.c2[j] : (cls == 0 ? -INFINITY : 0.f), (float)cls);
        }
        part += Bh[j] * Bh[j];
    }
    // block reduction helper
    auto bsum = [&](double v) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        __syncthreads();
        return t;
    };
    double Nmax = sqrt(bsum(part)) * (1.0 + 1e-6);
    double Emax = (double)Q.kvec[1] + u24 * Nmax;
    // The classes serve both passes (one-term and split): every bound below is the
    // larger of the two passes' bounds.
    for (int l = 2; l < L; ++l) {
        const TcLayer& ly = P.ly[l];
        const int K = ly.K, N = ly.N;
        const double Rmax = uq * Nmax + sqrt((double)K) * 0x1p-25;
        const double Lmax = uq * Nmax;
        const double u1 = K * (double)P.acc_unit, u3 = 3.0 * K * (double)P.acc_unit;
        const double Pa1 = Rmax + Emax + u1 * (Nmax + Rmax);
        const double Pa3 = Rmax + Emax + 0x1p-7 * Lmax + u3 * (Nmax + Rmax + 2.0 * Lmax);
        const double Pb = Nmax + Emax;
        __shared__ double Bn[1024];
        double part2 = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const float* Wr = net.W[l] + (size_t)i * K;
            double acc = 0.0;
            for (int j = 0; j < K; ++j) acc += fabs((double)Wr[j]) * Bh[j];
            const double em = fmax((double)ly.a[i] * Pa1 + (double)ly.b1[i] * Pb,
                                   (double)ly.a[i] * Pa3 + (double)ly.b3[i] * Pb);
            const double B = (acc * (1.0 + 1e-6) + em);
            const int gi = net.noff[l] + i;
            const double ub = Q.ub[gi];
            const bool cross = !(fabs(ub) > (B + (double)Q.thr[gi]) * (1.0 + 1e-6) + 4.0 * kTau);
            if (!cross)
                atomicOr(ub >= 0.0 ? &Q.cpos[l * 32 + (i >> 5)] : &Q.cneg[l * 32 + (i >> 5)], 1u << (i & 31));
            Bn[i] = (!cross && ub < 0.0) ? 0.0 : B;
            if (Q.kcol) {
                const int cls = cross ? 2 : (ub >= 0.0 ? 0 : 1);
                Q.kcol[2 * gi] = make_float4(Q.ub32[gi], ly.a[i], ly.b1[i], ly.b3[i]);
                Q.kcol[2 * gi + 1] = make_float4(Q.thr[gi], cls == 2 ? Q.c1[gi] : (cls == 0 ? 0.f : -INFINITY),
                                                 cls == 2 ? Q.c2[gi] : (cls == 0 ? -INFINITY : 0.f), (float)cls);
            }
            part2 += Bn[i] * Bn[i];
        }
        __syncthreads();
        const double E1 = ly.sq * Rmax + ly.sd1 * Nmax + (ly.sq + ly.sd1) * Emax + u1 * ly.fq * (Nmax + Rmax);
        const double E3 = ly.sa * Rmax + ly.sd3 * Nmax + (ly.sa + ly.sd3) * Emax + (double)ly.sl * Lmax +
                          u3 * ly.fq * (Nmax + Rmax + 2.0 * Lmax);
        double El = fmax(E1, E3) + (double)Q.kvec[l];
        Nmax = sqrt(bsum(part2)) * (1.0 + 1e-6);
        El += u24 * Nmax;
        Emax = El * (1.0 + 1e-6);
        for (int i = threadIdx.x; i < N; i += blockDim.x) Bh[i] = Bn[i];
        __syncthreads();
    }
}

// Compacted columns of one query (after k_classes_tc). For every hidden layer l
// the neurons not of the class "neg" get positions 0 .. count-1 in neuron order
// (perm), padded with "neg" positions to a multiple of 64 (kc[l]; kc[kMaxL+1+l]
// = count). A "neg" neuron's output change is 0 at every point of the box, so
// its column of the next layer's operand is all zeros: the dense layers run over
// the kept columns only, with the same products. Also the layer-1 tables and the
// s weight rows of layer 1 in compacted column order.
__global__ void __launch_bounds__(512) k_compact_perm(const __grid_constant__ TcParams P, NetView net,
                                                      QueryView* qs) {
    QueryView& Q = qs[0];
    __shared__ int wsum[16];
    __shared__ int cnt1_s, kc1_s;
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    for (int l = 1; l < P.L; ++l) {
        const int H = net.dims[l];  // <= 512 on the fused path
        const bool keep = t < H && !((Q.cneg[l * 32 + (t >> 5)] >> (t & 31)) & 1u);
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wsum[wp] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < 16; ++w) {
            if (w < wp) before += wsum[w];
            total += wsum[w];
        }
        const int kcl = max(64, (total + 63) & ~63);
        if (keep) {
            const int pos = before + __popc(m & ((1u << lane) - 1u));
            Q.perm[net.noff[l] + pos] = t;
            Q.kcolc[2 * (net.noff[l] + pos)] = Q.kcol[2 * (net.noff[l] + t)];
            Q.kcolc[2 * (net.noff[l] + pos) + 1] = Q.kcol[2 * (net.noff[l] + t) + 1];
        }
        if (t >= total && t < kcl) {  // padding: "neg" by position
            Q.perm[net.noff[l] + t] = 0;
            Q.kcolc[2 * (net.noff[l] + t)] = make_float4(0.f, 0.f, 0.f, 0.f);
            Q.kcolc[2 * (net.noff[l] + t) + 1] = make_float4(0.f, -INFINITY, 0.f, 1.f);
        }
        if (t == 0) {
            Q.compact = 1;
            Q.kc[l] = kcl;
            Q.kc[kMaxL + 1 + l] = total;
            if (l == 1) {
                cnt1_s = total;
                kc1_s = kcl;
            }
        }
        __syncthreads();
    }
    const int H1 = net.dims[1], cnt1 = cnt1_s, kc1 = kc1_s;
    for (int e = t; e < Q.s * Q.R * kc1; e += blockDim.x) {
        const int row = e / kc1, j = e - row * kc1;
        Q.tabc[(size_t)row * H1 + j] = j < cnt1 ? Q.tab[(size_t)row * H1 + Q.perm[j]] : 0.f;
    }
    for (int e = t; e < Q.s * kc1; e += blockDim.x) {
        const int p = e / kc1, j = e - p * kc1;
        Q.w1c[(size_t)p * H1 + j] = j < cnt1 ? net.WT[1][(size_t)Q.pix[p] * H1 + Q.perm[j]] : 0.f;
    }
}

struct CompactDst {
    void* wq[kTcMaxL + 1];
    void* wlo[kTcMaxL + 1];
};

// The query's copies of Wq_l and Wlo_l (l >= 2): row n' = neuron perm_l[n'] of
// layer l (the output layer keeps its rows), column k' = input perm_{l-1}[k'];
// zeros at padding positions. Same [Npad][K] layout as the net's copies.
__global__ void k_compact_gather(const __grid_constant__ TcParams P, NetView net, const QueryView* qs,
                                 CompactDst dst) {
    const QueryView& Q = qs[0];
    const int l = 2 + (int)blockIdx.y;
    if (l > P.L) return;
    const TcLayer& ly = P.ly[l];
    const int K = ly.K;
    const bool out = l == P.L;
    const int kin = Q.kc[l - 1], cin = Q.kc[kMaxL + l];
    const int rows = out ? ly.Npad : Q.kc[l];
    const int cout = out ? ly.Npad : Q.kc[kMaxL + 1 + l];
    const uint16_t* sq = static_cast<const uint16_t*>(ly.wq);
    const uint16_t* sl = static_cast<const uint16_t*>(ly.wlo);
    uint16_t* dq = static_cast<uint16_t*>(dst.wq[l]);
    uint16_t* dl = static_cast<uint16_t*>(dst.wlo[l]);
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int ro = r < cout ? (out ? r : Q.perm[net.noff[l] + r]) : -1;
        for (int k = threadIdx.x; k < kin; k += blockDim.x) {
            uint16_t a = 0, b = 0;  // +0 in both 16-bit formats
            if (ro >= 0 && k < cin) {
                const int ko = Q.perm[net.noff[l - 1] + k];
                a = sq[(size_t)ro * K + ko];
                b = sl[(size_t)ro * K + ko];
            }
            dq[(size_t)r * K + k] = a;
            dl[(size_t)r * K + k] = b;
        }
    }
    // the FP32 transposed copy for the FP32 pass: wtc[l][k'][n'] (row stride N)
    const int N = ly.N;
    const int ncols = out ? N : Q.kc[l];
    const int ncnt = out ? N : Q.kc[kMaxL + 1 + l];
    float* wt = Q.wtc[l];
    for (int k = blockIdx.x; k < kin; k += gridDim.x) {
        const int ko = k < cin ? Q.perm[net.noff[l - 1] + k] : -1;
        for (int n = threadIdx.x; n < ncols; n += blockDim.x) {
            const int no = n < ncnt ? (out ? n : Q.perm[net.noff[l] + n]) : -1;
            wt[(size_t)k * N + n] = (ko >= 0 && no >= 0) ? net.WT[l][(size_t)ko * N + no] : 0.f;
        }
    }
}

// ------------------------------------------------ kind::f16 accumulator probe
//
// One 128 x 128 tile with K = 256 (four 64-column chunks, the tensor screen's
// K-major 128-byte-swizzle layout) through TMA, tcgen05.mma kind::f16 and
// tcgen05.ld, exactly as the screen issues them. The host compares every output
// with its exact value (see tc_f16_selftest).
constexpr int ST_DIM = 128, ST_KCH = 4;

__global__ void __launch_bounds__(128, 1)
k_tc_selftest(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int bf,
              float* out, int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t* sa = base;                            // ST_KCH chunks of 128 rows x 128 bytes
    uint8_t* sb = base + ST_KCH * ST_DIM * 128;
    __shared__ unsigned long long bars[2];
    __shared__ uint32_t slot;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        tc::mbar_init(tc::smem_u32(&bars[0]), 1);
        tc::mbar_init(tc::smem_u32(&bars[1]), 1);
        abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&slot), ST_DIM);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = slot;
    if (threadIdx.x == 0) {
        tc::mbar_expect_tx(tc::smem_u32(&bars[0]), (uint32_t)(2 * ST_KCH * ST_DIM * 128));
        for (int c = 0; c < ST_KCH; ++c) {
            tc::tma_load_2d(tc::smem_u32(sa + c * ST_DIM * 128), &ta, 64 * c, 0, tc::smem_u32(&bars[0]));
            tc::tma_load_2d(tc::smem_u32(sb + c * ST_DIM * 128), &tb, 64 * c, 0, tc::smem_u32(&bars[0]));
        }
        bool ok = tc::mbar_wait(tc::smem_u32(&bars[0]), 0, &abort_flag);
        if (ok) {
            tc::tc_fence_after();
            const uint32_t idesc = tc::idesc_f16(ST_DIM, ST_DIM, bf != 0);
            for (int c = 0; c < ST_KCH; ++c)
                for (int ks = 0; ks < 4; ++ks)
                    tc::mma_f16(tmem, tc::desc_sw128(tc::smem_u32(sa + c * ST_DIM * 128) + ks * 32),
                                tc::desc_sw128(tc::smem_u32(sb + c * ST_DIM * 128) + ks * 32), idesc,
                                (c | ks) != 0);
        }
        // the commit also covers the case where nothing was issued
        tc::mma_commit(tc::smem_u32(&bars[1]));
        if (!tc::mbar_wait(tc::smem_u32(&bars[1]), 0, &abort_flag)) ok = false;
        if (!ok) atomicExch(status, 2);
    }
    __syncthreads();
    tc::tc_fence_after();
    if (!abort_flag) {
        const int lane = threadIdx.x & 31;
        for (int c = 0; c < ST_DIM; c += 32) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
            for (int e = 0; e < 32; ++e) out[(size_t)(32 * warp + lane) * ST_DIM + c + e] = v[e];
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, ST_DIM);
    }
}

// ------------------------------------------------------- host-side set-up

float up_f(double x) {
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, INFINITY);
    return f;
}

template <bool BF>
float q16(float x) {
    if (BF) return __bfloat162float(__float2bfloat16_rn(x));
    return __half2float(__float2half_rn(x));
}

}  // namespace

// The kind::f16 accumulator self-test (BF16 or FP16 operands, FP32 accumulate).
// The screens' bounds take the accumulation error of a K-term MMA dot product
// as at most K u sum_k |a_k b_k| with u = 2^-22 (an FP32 accumulator, whatever
// the order of its additions). The PTX ISA does not specify how the MMA rounds
// its partial sums, so the unit is measured here on the operand layout the
// screen uses, K = 256 over four K chunks:
//   - rows and columns 0..95: integers in [-2, 2]; products and sums are exact
//     in any accumulator, so a wrong value means a wrong layout (unsupported);
//   - five probe outputs whose exact sums need 17 to 24 significand bits (one
//     large product and 255 small ones of the same or the opposite sign, the
//     large one first or in the third chunk): exact in an FP32 accumulator,
//     so a short accumulator or one that truncates the small terms fails them;
//   - every other output (random operands m 2^e, 8-bit m, |value| in [2^-14, 4), random
//     signs, against the integer and probe rows and columns) must lie within
//     the model K 2^-22 sum |products| of its FP64 value.
// *unit = 2^-22 when all of these hold; 2^-13 when only the integers are exact
// and every output lies within K 2^-13 sum |products|; otherwise the screens are
// unsupported on this device. *worst = the largest |error| / (K sum |products|)
// seen over the tile (0 when every output is exact); *failed = bit i set when
// probe i (rows 127 down to 123) did not come back exact. The result is kept per
// device and operand type.
vbmc_status tc_f16_selftest(bool bf, float* unit, double* worst, int* failed) {
    static std::mutex mu;
    static int done[64][2] = {};
    static float units[64][2];
    static double worsts[64][2];
    static int fails[64][2];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return VBMC_ERR_CUDA;
    std::lock_guard<std::mutex> lk(mu);
    const int ti = bf ? 0 : 1;
    if (done[dev][ti]) {
        *unit = units[dev][ti];
        if (worst) *worst = worsts[dev][ti];
        if (failed) *failed = fails[dev][ti];
        return VBMC_OK;
    }
    constexpr int Kt = 64 * ST_KCH;
    std::vector<uint16_t> ha((size_t)ST_DIM * Kt), hb((size_t)ST_DIM * Kt);
    std::vector<double> va(ha.size()), vb(hb.size());
    auto bits = [&](double x) -> uint16_t {
        const float f = (float)x;
        if (bf) {
            __nv_bfloat16 h = __float2bfloat16_rn(f);
            return *reinterpret_cast<uint16_t*>(&h);
        }
        __half h = __float2half_rn(f);
        return *reinterpret_cast<uint16_t*>(&h);
    };
    auto put = [&](std::vector<uint16_t>& h, std::vector<double>& v, int r, int k, double x) {
        h[(size_t)r * Kt + k] = bits(x);
        v[(size_t)r * Kt + k] = x;  // every value below is exact in both formats
    };
    uint64_t z = 0x243F6A8885A308D3ull;  // SplitMix64 stream for the random operands
    auto rnd = [&]() {
        z += 0x9E3779B97F4A7C15ull;
        uint64_t x = z;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        return x ^ (x >> 31);
    };
    auto random_value = [&]() {
        const uint64_t r = rnd();
        const double m = (double)(128 + (r & 127));      // 8 significand bits
        const int e = (int)((r >> 8) % 16) - 21;          // m 2^e in [2^-14, 2^2): normal in FP16
        return ((r >> 20) & 1 ? -1.0 : 1.0) * std::ldexp(m, e);
    };
    for (int r = 0; r < ST_DIM; ++r)
        for (int k = 0; k < Kt; ++k) {
            if (r < 96) {
                put(ha, va, r, k, (double)((int)((r * 7 + k * 3 + 1) % 5) - 2));
                put(hb, vb, r, k, (double)((int)((r * 11 + k * 5 + 2) % 5) - 2));
            } else {
                put(ha, va, r, k, random_value());
                put(hb, vb, r, k, random_value());
            }
        }
    // probe rows r of A and B: products p_0 = a0 b0 at position k0, and 255 small
    // products q = as bs; the exact sums fit 24 significand bits
    struct Probe { int r, k0; double a0, b0, as, bs; };
    const Probe probes[5] = {
        {127, 0, 1.0, 1.0, 0x1p-12, 0x1p-11},      // 1 + 255 2^-23
        {126, 0, 16.0, 16.0, 0x1p-8, 0x1p-7},      // 256 + 255 2^-15
        {125, 0, -1.0, 1.0, 0x1p-12, 0x1p-11},     // -1 + 255 2^-23
        {124, 128, 1.0, 1.0, 0x1p-12, 0x1p-11},    // 128 2^-23, then 1, then 127 2^-23
        {123, 0, 4.0, 2.0, 0x1p-10, 0x1p-10},      // 8 + 255 2^-20
    };
    for (const Probe& p : probes)
        for (int k = 0; k < Kt; ++k) {
            put(ha, va, p.r, k, k == p.k0 ? p.a0 : p.as);
            put(hb, vb, p.r, k, k == p.k0 ? p.b0 : p.bs);
        }
    void *da = nullptr, *db = nullptr;
    float* dout = nullptr;
    int* dst = nullptr;
    vbmc_status res = VBMC_ERR_CUDA;
    std::vector<float> got((size_t)ST_DIM * ST_DIM);
    int status = 0;
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    cudaDriverEntryPointQueryResult qr;
    CUtensorMap ta, tb;
    const CUtensorMapDataType dt = bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    cuuint64_t gdim[2] = {(cuuint64_t)Kt, (cuuint64_t)ST_DIM};
    cuuint64_t gstr[1] = {(cuuint64_t)Kt * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)ST_DIM};
    cuuint32_t estr[2] = {1, 1};
    const size_t smem = (size_t)2 * ST_KCH * ST_DIM * 128 + 1024;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&encode, 12000, cudaEnableDefault,
                                         &qr) != cudaSuccess || !encode)
        goto done;
    if (cudaMalloc(&da, 2 * ha.size()) != cudaSuccess || cudaMalloc(&db, 2 * hb.size()) != cudaSuccess ||
        cudaMalloc(&dout, sizeof(float) * got.size()) != cudaSuccess || cudaMalloc(&dst, sizeof(int)) != cudaSuccess)
        goto done;
    if (cudaMemcpy(da, ha.data(), 2 * ha.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(db, hb.data(), 2 * hb.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(dst, 0, sizeof(int)) != cudaSuccess)
        goto done;
    if (encode(&ta, dt, 2, da, gdim, gstr, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        encode(&tb, dt, 2, db, gdim, gstr, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        goto done;
    cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_tc_selftest<<<1, 128, smem>>>(ta, tb, bf ? 1 : 0, dout, dst);
    if (cudaDeviceSynchronize() != cudaSuccess) goto done;
    if (cudaMemcpy(got.data(), dout, sizeof(float) * got.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&status, dst, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        goto done;
    if (status != 0) {
        res = VBMC_ERR_DEVICE;
        goto done;
    }
    {
        bool layout_ok = true;
        int probe_fail = 0;
        double w = 0.0;
        for (int r = 0; r < ST_DIM; ++r)
            for (int n = 0; n < ST_DIM; ++n) {
                double ex = 0.0, mag = 0.0;
                for (int k = 0; k < Kt; ++k) {
                    const double p = va[(size_t)r * Kt + k] * vb[(size_t)n * Kt + k];
                    ex += p;  // products of 8- and 11-bit values: exact, sums within FP64
                    mag += std::fabs(p);
                }
                const double g = (double)got[(size_t)r * ST_DIM + n];
                const double err = std::fabs(g - ex);
                if (r < 96 && n < 96) {
                    if (err != 0.0) layout_ok = false;
                    continue;
                }
                if (r == n && r >= 123 && err != 0.0) probe_fail |= 1 << (127 - r);
                if (mag > 0.0) w = std::max(w, err / ((double)Kt * mag));
                else if (err != 0.0) w = INFINITY;
            }
        if (!layout_ok) {
            res = VBMC_ERR_UNSUPPORTED;
            goto done;
        }
        float u = 0.f;
        if (!probe_fail && w <= 0x1p-22) u = 0x1p-22f;
        else if (w <= 0x1p-13) u = 0x1p-13f;
        if (u == 0.f) {
            res = VBMC_ERR_UNSUPPORTED;
            goto done;
        }
        units[dev][ti] = u;
        worsts[dev][ti] = w;
        fails[dev][ti] = probe_fail;
        done[dev][ti] = 1;
        *unit = u;
        if (worst) *worst = w;
        if (failed) *failed = probe_fail;
        res = VBMC_OK;
    }
done:
    cudaFree(da);
    cudaFree(db);
    cudaFree(dout);
    cudaFree(dst);
    return res;
}

bool tc_supported(const NetView& v, int precision) {
    if (precision != VBMC_PREC_BF16 && precision != VBMC_PREC_FP16) return false;
    if (v.act != ACT_RELU || v.L < 2 || v.L > kTcMaxL) return false;
    if (v.dims[1] % 64 || v.dims[1] > 512) return false;
    for (int l = 2; l < v.L; ++l)
        if (v.dims[l] % 64 || v.dims[l] > 512) return false;
    if (v.dims[v.L] > kTcMaxOut) return false;
    if (v.flip_words > 256) return false;
    // a layer l >= 3 wider than 64 reuses the accumulator columns of layer l-1, so
    // its MMAs start only after layer l-1 is drained: the drain must fit the
    // operand ring (at most NA chunks of 64)
    for (int l = 3; l <= v.L; ++l) {
        const int Npad = l == v.L ? (v.dims[l] <= 16 ? 16 : 32) : v.dims[l];
        if (Npad > 64 && v.dims[l - 1] / 64 > NA) return false;
    }
    return true;
}

template <bool BF>
static vbmc_status build_prec(TcNet& tc, const NetView& v, const std::vector<std::vector<float>>& W,
                              TcParams& P) {
    using T = typename std::conditional<BF, __nv_bfloat16, __half>::type;
    std::memset(&P, 0, sizeof(P));
    (void)cudaGetLastError();  // start from a clean error state
    P.L = v.L;
    P.bf16 = BF ? 1 : 0;
    {
        const vbmc_status ss = tc_f16_selftest(BF, &P.acc_unit, nullptr, nullptr);
        if (ss != VBMC_OK) return ss;
    }
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&encode, 12000,
                                         cudaEnableDefault, &qr) !=
            cudaSuccess ||
        !encode)
        return VBMC_ERR_CUDA;
    for (int l = 2; l <= v.L; ++l) {
        const int K = v.dims[l - 1], N = v.dims[l];
        const bool out = (l == v.L);
        const int Npad = out ? (N <= 16 ? 16 : 32) : N;
        TcLayer& ly = P.ly[l];
        ly.K = K;
        ly.N = N;
        ly.Npad = Npad;
        ly.slice = std::min(Npad, 128);  // one 16 KB weight slot per N slice
        ly.nslice = Npad / ly.slice;
        ly.kch = K / 64;
        std::vector<T> hq((size_t)Npad * K), hlo((size_t)Npad * K);
        std::vector<double> Wq((size_t)N * K), Wd1((size_t)N * K), Wd3((size_t)N * K), Wa((size_t)N * K),
            Wl((size_t)N * K);
        std::vector<float> a(Npad, 0.f), b1(Npad, 0.f), b3(Npad, 0.f);
        double fq2 = 0.0;
        for (int i = 0; i < Npad; ++i) {
            double a2 = 0.0, d12 = 0.0, d32 = 0.0;
            for (int j = 0; j < K; ++j) {
                const float w = i < N ? W[l][(size_t)i * K + j] : 0.f;
                const float wq = q16<BF>(w);
                const float wl = q16<BF>(w - wq);
                hq[(size_t)i * K + j] = BF ? (T)__float2bfloat16_rn(wq) : (T)__float2half_rn(wq);
                hlo[(size_t)i * K + j] = BF ? (T)__float2bfloat16_rn(wl) : (T)__float2half_rn(wl);
                if (i < N) {
                    const double wa = (double)wq + (double)wl;
                    Wq[(size_t)i * K + j] = wq;
                    Wd1[(size_t)i * K + j] = (double)w - wq;
                    Wd3[(size_t)i * K + j] = (double)w - wa;
                    Wa[(size_t)i * K + j] = wa;
                    Wl[(size_t)i * K + j] = wl;
                }
                a2 += (double)wq * wq;
                d12 += ((double)w - wq) * ((double)w - wq);
                d32 += ((double)w - wq - wl) * ((double)w - wq - wl);
            }
            fq2 += a2;
            // split mode uses ||Wq + Wlo|| <= ||Wq|| + ||Wlo||; bound with 1 + 2^-7
            a[i] = up_f(std::sqrt(a2) * (1.0 + 0x1p-7) * (1.0 + 1e-9));
            b1[i] = up_f(std::sqrt(d12) * (1.0 + 1e-9));
            b3[i] = up_f(std::sqrt(d32) * (1.0 + 1e-9));
        }
        ly.fq = up_f(std::sqrt(fq2) * (1.0 + 0x1p-7) * (1.0 + 1e-9));
        // ||Wlo_i|| <= 2^-7 ||Wq_i|| (checked: the split bound relies on it)
        for (int i = 0; i < N; ++i) {
            double l2 = 0.0, q2 = 0.0;
            for (int j = 0; j < K; ++j) {
                l2 += Wl[(size_t)i * K + j] * Wl[(size_t)i * K + j];
                q2 += Wq[(size_t)i * K + j] * Wq[(size_t)i * K + j];
            }
            if (l2 > 0x1p-14 * q2 * (1.0 + 1e-9)) return VBMC_ERR_UNSUPPORTED;
        }
        if (!out) {
            ly.sq = up_f(spectral_bound(Wq, N, K));
            ly.sa = up_f(spectral_bound(Wa, N, K));
            ly.sl = up_f(spectral_bound(Wl, N, K));
            ly.sd1 = up_f(spectral_bound(Wd1, N, K));
            ly.sd3 = up_f(spectral_bound(Wd3, N, K));
            if (!(ly.sq > 0.f) || !(ly.sa > 0.f)) return VBMC_ERR_CUDA;
        } else {
            // pair constants for the margin: ||Wa_D - Wa_o||, ||Wr_D - Wr_o|| (1x: b1 rows,
            // split: b3 rows), ||W_D - W_o||, ||Wlo_D - Wlo_o||, a_D + a_o
            std::vector<float> pair((size_t)N * N * 5, 0.f);
            for (int D = 0; D < N; ++D)
                for (int o = 0; o < N; ++o) {
                    double A2 = 0.0, B12 = 0.0, B32 = 0.0, C2 = 0.0, L2 = 0.0, Q2 = 0.0;
                    for (int j = 0; j < K; ++j) {
                        const double wD = W[l][(size_t)D * K + j], wo = W[l][(size_t)o * K + j];
                        const double dq = Wq[(size_t)D * K + j] - Wq[(size_t)o * K + j];
                        const double da = Wa[(size_t)D * K + j] - Wa[(size_t)o * K + j];
                        const double d1 = Wd1[(size_t)D * K + j] - Wd1[(size_t)o * K + j];
                        const double d3 = Wd3[(size_t)D * K + j] - Wd3[(size_t)o * K + j];
                        const double dl = Wl[(size_t)D * K + j] - Wl[(size_t)o * K + j];
                        Q2 += dq * dq;
                        A2 += da * da;
                        B12 += d1 * d1;
                        B32 += d3 * d3;
                        C2 += (wD - wo) * (wD - wo);
                        L2 += dl * dl;
                    }
                    float* c = &pair[((size_t)D * N + o) * 5];
                    (void)B32;
                    c[0] = up_f(std::sqrt(std::max(Q2, A2)) * (1.0 + 1e-9));
                    c[1] = up_f(std::sqrt(std::max(B12, B32)) * (1.0 + 1e-9));
                    c[2] = up_f(std::sqrt(C2) * (1.0 + 1e-9));
                    c[3] = up_f(std::sqrt(L2) * (1.0 + 1e-9));
                    c[4] = up_f(((double)a[D] + (double)a[o]) * (1.0 + 1e-9));
                }
            float* dp = nullptr;
            if (cudaMalloc(&dp, sizeof(float) * pair.size()) != cudaSuccess) return VBMC_ERR_OOM;
            tc.owned.push_back(dp);
            cudaMemcpy(dp, pair.data(), sizeof(float) * pair.size(), cudaMemcpyHostToDevice);
            P.pair = dp;
        }
        // device copies
        T *dq = nullptr, *dl = nullptr;
        float *da = nullptr, *db1 = nullptr, *db3 = nullptr;
        if (cudaMalloc(&dq, sizeof(T) * hq.size()) != cudaSuccess) return VBMC_ERR_OOM;
        tc.owned.push_back(dq);
        if (cudaMalloc(&dl, sizeof(T) * hlo.size()) != cudaSuccess) return VBMC_ERR_OOM;
        tc.owned.push_back(dl);
        if (cudaMalloc(&da, sizeof(float) * Npad) != cudaSuccess) return VBMC_ERR_OOM;
        tc.owned.push_back(da);
        if (cudaMalloc(&db1, sizeof(float) * Npad) != cudaSuccess) return VBMC_ERR_OOM;
        tc.owned.push_back(db1);
        if (cudaMalloc(&db3, sizeof(float) * Npad) != cudaSuccess) return VBMC_ERR_OOM;
        tc.owned.push_back(db3);
        cudaMemcpy(dq, hq.data(), sizeof(T) * hq.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(dl, hlo.data(), sizeof(T) * hlo.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(da, a.data(), sizeof(float) * Npad, cudaMemcpyHostToDevice);
        cudaMemcpy(db1, b1.data(), sizeof(float) * Npad, cudaMemcpyHostToDevice);
        cudaMemcpy(db3, b3.data(), sizeof(float) * Npad, cudaMemcpyHostToDevice);
        ly.a = da;
        ly.b1 = db1;
        ly.b3 = db3;
        ly.wq = dq;
        ly.wlo = dl;
        const CUtensorMapDataType dt = BF ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
        cuuint64_t gdim[2] = {(cuuint64_t)K, (cuuint64_t)Npad};
        cuuint64_t gstr[1] = {(cuuint64_t)K * 2};
        cuuint32_t box[2] = {64, (cuuint32_t)ly.slice};
        cuuint32_t estr[2] = {1, 1};
        CUresult e1 = encode(&P.tq[l], dt, 2, dq, gdim, gstr, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        CUresult e2 = encode(&P.tlo[l], dt, 2, dl, gdim, gstr, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (e1 != CUDA_SUCCESS || e2 != CUDA_SUCCESS) return VBMC_ERR_CUDA;
    }
    if (cudaGetLastError() != cudaSuccess) return VBMC_ERR_CUDA;
    return VBMC_OK;
}

vbmc_status tc_build(TcNet& tc, const NetView& v, const std::vector<std::vector<float>>& W,
                     const std::vector<std::vector<float>>&, int precision) {
    const int pi = precision == VBMC_PREC_BF16 ? 0 : 1;
    if (tc.prec[pi].ready) return VBMC_OK;
    vbmc_status st = pi == 0 ? build_prec<true>(tc, v, W, tc.prec[pi].p)
                             : build_prec<false>(tc, v, W, tc.prec[pi].p);
    if (st == VBMC_OK) tc.prec[pi].ready = true;
    return st;
}

void tc_free(TcNet& tc) {
    for (void* p : tc.owned) cudaFree(p);
    tc.owned.clear();
    tc.prec[0].ready = tc.prec[1].ready = false;
}

vbmc_status tc_query_work_alloc(TcQueryWork& w, const NetView& v) {
    for (int l = 2; l <= v.L; ++l) {
        const int K = v.dims[l - 1], N = v.dims[l];
        const int Npad = l == v.L ? (N <= 16 ? 16 : 32) : N;
        for (void** pp : {&w.wq[l], &w.wlo[l]}) {
            if (cudaMalloc(pp, (size_t)2 * Npad * K) != cudaSuccess) {
                tc_query_work_free(w);
                return VBMC_ERR_OOM;
            }
            w.owned.push_back(*pp);
        }
    }
    return VBMC_OK;
}

void tc_query_work_free(TcQueryWork& w) {
    for (void* p : w.owned) cudaFree(p);
    w.owned.clear();
    for (int l = 0; l <= kTcMaxL; ++l) w.wq[l] = w.wlo[l] = nullptr;
    w.maps[0] = w.maps[1] = false;
}

void tc_launch_query_setup(TcNet& tc, const NetView& v, QueryView* d_q, int nq, int precision,
                           cudaStream_t st, TcQueryWork* qw) {
    const TcParams& P = tc.prec[precision == VBMC_PREC_BF16 ? 0 : 1].p;
    k_classes_tc<<<nq, 512, 0, st>>>(P, v, d_q);
    if (qw && nq == 1) {
        k_compact_perm<<<1, 512, 0, st>>>(P, v, d_q);
        CompactDst dst{};
        for (int l = 2; l <= v.L; ++l) {
            dst.wq[l] = qw->wq[l];
            dst.wlo[l] = qw->wlo[l];
        }
        k_compact_gather<<<dim3(128, (unsigned)(v.L - 1)), 256, 0, st>>>(P, v, d_q, dst);
    }
}

namespace {

// Kernel parameters of a compacted call: the net's, with the weight maps of
// the query's own copies and 128-row slices for the hidden layers.
bool compact_params(const TcParams& P, const NetView& v, TcQueryWork& qw, int pi, TcParams& out) {
    if (!qw.maps[pi]) {
        PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&encode, 12000, cudaEnableDefault,
                                             &qr) != cudaSuccess || !encode)
            return false;
        const CUtensorMapDataType dt = pi == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
        for (int l = 2; l <= v.L; ++l) {
            const TcLayer& ly = P.ly[l];
            const int slice = l == v.L ? ly.slice : 128;
            cuuint64_t gdim[2] = {(cuuint64_t)ly.K, (cuuint64_t)ly.Npad};
            cuuint64_t gstr[1] = {(cuuint64_t)ly.K * 2};
            cuuint32_t box[2] = {64, (cuuint32_t)slice};
            cuuint32_t estr[2] = {1, 1};
            if (encode(&qw.tq[pi][l], dt, 2, qw.wq[l], gdim, gstr, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
                encode(&qw.tlo[pi][l], dt, 2, qw.wlo[l], gdim, gstr, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return false;
        }
        qw.maps[pi] = true;
    }
    out = P;
    out.compact = 1;
    for (int l = 2; l <= v.L; ++l) {
        out.tq[l] = qw.tq[pi][l];
        out.tlo[l] = qw.tlo[pi][l];
        if (l < v.L) out.ly[l].slice = 128;
    }
    return true;
}

}  // namespace

template <bool SPLIT, bool BF>
static void launch_k(const TcParams& P, const NetView& v, const QueryView* d_q, int nq,
                     const unsigned long long* tp, unsigned long long ntiles, const QEntry* g,
                     const unsigned long long* gc, unsigned long long cap, Queue out, int level,
                     int n_sm, cudaStream_t st, unsigned long long* claim) {
    const size_t smem = sizeof(TcSmem) + 1024;
    auto kern = k_tc<SPLIT, BF>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    unsigned grid = (unsigned)n_sm;
    if (!g && ntiles < grid) grid = (unsigned)(ntiles ? ntiles : 1);
    kern<<<grid, TC_THREADS, smem, st>>>(P, v, d_q, nq, tp, g, gc, cap, out, level, claim);
}

vbmc_status tc_launch_screen(TcNet& tc, const NetView& v, const QueryView* d_q, int nq,
                             const unsigned long long* d_tile_prefix, unsigned long long ntiles,
                             int precision, Queue out, int out_level, int n_sm, cudaStream_t st,
                             TcQueryWork* qw, unsigned long long* d_claim) {
    const bool bf = precision == VBMC_PREC_BF16;
    TcParams Pc;
    if (qw && nq == 1 && !compact_params(tc.prec[bf ? 0 : 1].p, v, *qw, bf ? 0 : 1, Pc)) return VBMC_ERR_CUDA;
    const TcParams& P = (qw && nq == 1) ? Pc : tc.prec[bf ? 0 : 1].p;
    if (d_claim && cudaMemsetAsync(d_claim, 0, sizeof(unsigned long long), st) != cudaSuccess) return VBMC_ERR_CUDA;
    if (bf) launch_k<false, true>(P, v, d_q, nq, d_tile_prefix, ntiles, nullptr, nullptr, 0, out, out_level, n_sm, st, d_claim);
    else launch_k<false, false>(P, v, d_q, nq, d_tile_prefix, ntiles, nullptr, nullptr, 0, out, out_level, n_sm, st, d_claim);
    return cudaPeekAtLastError() == cudaSuccess ? VBMC_OK : VBMC_ERR_CUDA;  // the caller reports the error
}

vbmc_status tc_launch_gather(TcNet& tc, const NetView& v, const QueryView* d_q, const QEntry* in,
                             const unsigned long long* in_count, unsigned long long cap,
                             int precision, Queue out, int n_sm, cudaStream_t st, TcQueryWork* qw) {
    const bool bf = precision == VBMC_PREC_BF16;
    TcParams Pc;
    if (qw && !compact_params(tc.prec[bf ? 0 : 1].p, v, *qw, bf ? 0 : 1, Pc)) return VBMC_ERR_CUDA;
    const TcParams& P = qw ? Pc : tc.prec[bf ? 0 : 1].p;
    if (bf) launch_k<true, true>(P, v, d_q, 1, nullptr, 0, in, in_count, cap, out, 1, n_sm, st, nullptr);
    else launch_k<true, false>(P, v, d_q, 1, nullptr, 0, in, in_count, cap, out, 1, n_sm, st, nullptr);
    return cudaPeekAtLastError() == cudaSuccess ? VBMC_OK : VBMC_ERR_CUDA;  // the caller reports the error
}

int tc_tile_points() { return MROWS; }

}  // namespace vbmc
