// screen_simt.cuh -- the plain FP32 path on CUDA cores, with a proven error bound.
//
// A CTA owns a tile of MT points (8 warps x PPW points). For each point:
//   S1  decode t into s digits (first pixel most significant)
//   S2  layer 1 incrementally: du_j = sum_p W_1[j][pix_p] dv_p / 255   (Eq. 1)
//   S3  sign test and delta activation dh = act(ub + du) - act(ub)    (Eq. 2, sign)
//   S4  layers 2..L in FP32 on the deltas: du_l = W_l dh_{l-1}, weight
//       chunks staged in shared memory, 128 accumulators per thread
//   S5  logits, class, margin, adversarial flag                       (Eq. 10)
//   S6  certain sign changes -> flip mask; SS-Cover pairs of the point
//   S7  verdict bit, count, first witness; undecided points -> queue
//
// Error bound (per point, per layer, u = 2^-24, gamma_n = n u / (1 - n u)):
//   N_l = ||dh_l||_2 as computed (rounded up), E_l = bound on ||dh_l - exact||_2
//   X_l = gamma_{H_{l-1}} N_{l-1} + E_{l-1}
//   |du_l,i - exact| <= ||W_l,i||_2 X_l              (dot-product error + propagated error)
//   E_l = lambda (rho_l + sigma_l E_{l-1}) + kvec_l + u N_l
//         (lambda = 1 for ReLU, 1/4 for sigmoid), where rho_l bounds the l2 norm
//         of the layer's rounding errors: the a priori ||W_l||_F gamma N_{l-1},
//         or the a posteriori bound from checkpointed partial sums (dense_layer),
//         whichever is smaller; the output layer's per-output rounding is
//         bounded the same way.
// A neuron's sign is certain when |fl(ub) + du| exceeds that bound plus the
// constant threshold (fp32 rounding of ub, 2 tau); the verdict is certain
// when every margin difference exceeds the combined bound. Anything else
// sends the whole point to the next pass.
#pragma once
#include "dev.cuh"
#include "launch.h"

namespace vbmc {
namespace simt {

constexpr int KC = 8;
constexpr int FCAP = 6;
constexpr int THREADS = 256;

template <int PPW, int NQ>
struct SimtSmem {
    static constexpr int MT = 8 * PPW;
    static constexpr int HS = 32 * NQ;
    static constexpr int WS = HS + 4;
    float A[MT][HS + 4];  // rows padded by 16 bytes: float4 reads of 4 consecutive rows hit distinct banks
    float Wsm[2][KC][WS];
    unsigned long long t[MT];
    int q[MT];
    int valid[MT];
    int unc[MT];
    int vstate[MT];
    float N[MT];
    float E[MT];
    float rho[MT][32];  // output layer (width <= 32): rounding bound of each output
    int fcnt[MT][kMaxL + 1];
    short flist[MT][kMaxL + 1][FCAP];
    unsigned char dig[MT][kMaxS];
    unsigned long long g;  // the CTA's current tile
    float cpx[MT][kMaxS];  // per point and pixel: fl(dv_p / 255), the pixel's input change
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Upper bound of sqrt of a non-negative sum of <= 1024 fp32 terms computed in fp32.
__device__ __forceinline__ float norm_up(float s) {
    return __fsqrt_ru(__fmul_ru(s, 1.0002f));
}

__device__ __forceinline__ float act_delta(int act, float du, float u, float c1, float c2) {
    if (act == ACT_RELU) return fmaxf(du + c1, c2);
    if (act == ACT_SIGMOID) return 1.0f / (1.0f + expf(-u)) - c2;
    return du;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Neuron held in accumulator slot qq of a lane. With 4 or more slots per lane the
// lane holds groups of 4 consecutive neurons (128 g + 4 lane + e), so its weights
// of one k come in with 16-byte shared-memory loads (a warp's load covers 128
// contiguous bytes per phase: no bank conflicts); with one slot, neuron = lane.
template <int NQA>
__device__ __forceinline__ int slot_neuron(int lane, int qq) {
    return NQA >= 4 ? 128 * (qq >> 2) + 4 * lane + (qq & 3) : lane + 32 * qq;
}

// Sums of non-negative fp32 terms with every addition rounded up: an upper bound.
__device__ __forceinline__ float warp_sum_ru(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_ru(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One dense layer l >= 2 for the tile: du = W_l dh_{l-1} (FP32 FMA, sequential over
// k), then the sign tests, the delta activation and the per-point error terms.
// NQA = neuron slots per lane actually used (1 for narrow output layers).
//
// Rounding of the dot products, a priori: |err_i| <= gamma_K sum_j |W_ij x_j|.
// A posteriori, from the partial sums: each FMA's rounding error is at most u
// times its computed result s_k, so |err_i| <= u sum_k |s_k,i|. The sum is
// kept at checkpoints every CKL = CKC * KC terms (segment starts g): within a
// segment |s_k| <= (|s_g| + sum_{j in g} |t_j|) / (1 - CKL u), hence
//   |err_i| <= u' CKL (V_i + ||W_i|| ||x||),  V_i = sum_g |s_g,i|,
// u' = u / (1 - CKL u). Over the layer, ||V||_2 <= sqrt(G sum_g ||s_g||^2)
// (Cauchy-Schwarz over the G segments), which each lane accumulates for its
// neurons (one register per point); with one neuron per lane (narrow layers)
// V_i itself is kept. Both bounds hold; the smaller one is used.
constexpr int CKC = 2;                       // chunks per checkpoint segment
constexpr float kUseg = 0x1.00002p-24f * (float)(CKC * KC);  // u' CKL, rounded up

// Register-blocked dense layer (paired slot widths; the epilogue loads each
// column's constants once for a tile of one query, per point otherwise):
// lane = (point group pg of 4, column group ng of 8); each lane accumulates 4
// points x QL columns, warps split the tile into blocks of 16 points x CBW
// columns. A weight float4 is read by 8 distinct lanes (one 128-byte
// wavefront, broadcast to the 4 point groups) and an operand float4 by 4
// (padded rows: one wavefront), so the FMAs, not the shared-memory reads, set
// the pace. Per point and column the operations are those of dense_layer:
// the same FMA sequence over k, checkpoints, sign tests and delta activation;
// the per-point sums of squares are combined across lanes and warps in
// another order (bounds that hold for any order).
template <int PPW, int NQ, int NQA>
__device__ __forceinline__ void dense_blocked(SimtSmem<PPW, NQ>& S, const NetView& net,
                                              const QueryView* __restrict__ qs, int l, int warp, int lane,
                                              bool cmp, bool oneq) {
    const QueryView& Q = qs[0];  // compacted columns: one query (cmp implies oneq)
    constexpr int HS = SimtSmem<PPW, NQ>::HS;
    constexpr int MT = SimtSmem<PPW, NQ>::MT;
    constexpr int HW = 32 * NQA;
    constexpr int WSL = HW + 4;
    constexpr int KCL = KC;
    constexpr int NPB = PPW / 2;     // blocks of 16 points
    constexpr int NCB = 16 / PPW;    // column blocks per point block
    constexpr int CBW = HW / NCB;    // columns per block
    constexpr int QL = CBW / 8;      // columns per lane
    constexpr int QT = QL / 4;       // float4 groups per lane
    static_assert(NPB * NCB == 8 && QL % 4 == 0 && QL <= 32 && 3 * NCB <= 32, "blocked layout");
    const int L = net.L;
    const int NS = net.dims[l];
    const int K = cmp ? Q.kc[l - 1] : net.dims[l - 1];
    const int N = (cmp && l < L) ? Q.kc[l] : NS;
    const int cntN = (cmp && l < L) ? Q.kc[kMaxL + 1 + l] : NS;
    const float* __restrict__ WT = cmp ? Q.wtc[l] : net.WT[l];  // [K][NS]
    const int nchunks = (K + KCL - 1) / KCL;
    float* const Wb = &S.Wsm[0][0][0];
    const int pbk = warp % NPB, cb = warp / NPB;
    const int pg = lane >> 3, ng = lane & 7;
    const int colb = cb * CBW + 4 * ng;  // the lane's columns: colb + 32 t + e
    int mrow[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) mrow[i] = pbk * 16 + 4 * i + pg;
    float2 acc[4][QT][2];
    float chk[4];  // sum_g ||s_g||^2 over this lane's columns, per point
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        chk[i] = 0.f;
#pragma unroll
        for (int t = 0; t < QT; ++t) acc[i][t][0] = acc[i][t][1] = make_float2(0.f, 0.f);
    }
    const bool vec = (N % 4) == 0 && (NS % 4) == 0;
    auto load_chunk = [&](int c, int buf) {
        float* const dst = Wb + buf * (KCL * WSL);
        if (vec) {
            for (int e = threadIdx.x; e < KCL * (HW / 4); e += THREADS) {
                const int kk = e / (HW / 4), n = (e % (HW / 4)) * 4, k = c * KCL + kk;
                const bool ok = k < K && n < N;
                cp_async16(dst + kk * WSL + n, ok ? (const void*)&WT[(size_t)k * NS + n] : (const void*)WT, ok);
            }
        } else {
            for (int e = threadIdx.x; e < KCL * HW; e += THREADS) {
                const int kk = e / HW, n = e % HW, k = c * KCL + kk;
                const bool ok = k < K && n < N;
                cp_async4(dst + kk * WSL + n, ok ? (const void*)&WT[(size_t)k * NS + n] : (const void*)WT, ok);
            }
        }
        cp_async_commit();
    };
    __syncthreads();  // previous users of Wsm are done
    load_chunk(0, 0);
    for (int c = 0; c < nchunks; ++c) {
        const int buf = c & 1;
        cp_async_wait0();
        __syncthreads();  // chunk c visible to all; chunk c-1's buffer free
        if (c + 1 < nchunks) load_chunk(c + 1, buf ^ 1);
        const float* const wc = Wb + buf * (KCL * WSL);
#pragma unroll
        for (int kk = 0; kk < KCL; kk += 4) {
            const int k0 = c * KCL + kk;
            if (k0 > 0 && k0 % (CKC * KC) == 0) {  // checkpoint: the partial sums at k = k0
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int t = 0; t < QT; ++t)
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            chk[i] = __fmaf_ru(acc[i][t][h].x, acc[i][t][h].x, chk[i]);
                            chk[i] = __fmaf_ru(acc[i][t][h].y, acc[i][t][h].y, chk[i]);
                        }
            }
            float4 a4[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a4[i] = *reinterpret_cast<const float4*>(&S.A[mrow[i]][k0]);
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
#pragma unroll
                for (int t = 0; t < QT; ++t) {
                    const float4 w4 = *reinterpret_cast<const float4*>(wc + (kk + k4) * WSL + colb + 32 * t);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float av = k4 == 0 ? a4[i].x : k4 == 1 ? a4[i].y : k4 == 2 ? a4[i].z : a4[i].w;
                        const float2 aa = make_float2(av, av);
                        acc[i][t][0] = __ffma2_rn(aa, make_float2(w4.x, w4.y), acc[i][t][0]);
                        acc[i][t][1] = __ffma2_rn(aa, make_float2(w4.z, w4.w), acc[i][t][1]);
                    }
                }
            }
        }
    }
    __syncthreads();  // every warp has read this layer's operand rows: they are overwritten below
    // epilogue: the sign tests and delta activation of each (point, column)
    const float* rn = net.rownorm[l];
    const int off = net.noff[l];
    const float lf = net.lamfrob[l], gl = net.gam[l];
    const float lam = net.act == ACT_SIGMOID ? 0.25f : 1.0f;
    const float G = (float)((nchunks * KCL + CKC * KC - 1) / (CKC * KC));  // checkpoint segments
    unsigned vmask = 0u;
    float X[4], nsum[4], usum[4];
    uint32_t uncb[4], flipb[4];  // per slot: uncertain sign, certain change
    int qi[4];                   // each point's query
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        qi[i] = oneq ? 0 : S.q[mrow[i]];
        vmask |= (unsigned)(S.valid[mrow[i]] != 0) << i;
        X[i] = __fmaf_ru(gl, S.N[mrow[i]], S.E[mrow[i]]);
        nsum[i] = usum[i] = 0.f;
        uncb[i] = flipb[i] = 0u;
    }
#pragma unroll
    for (int t = 0; t < QT; ++t) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int n = colb + 32 * t + e;  // position
            const int slot = 4 * t + e;
            // neuron at position n; -1: a padding position (output change 0)
            const int no = (cmp && l < L) ? (n < cntN ? Q.perm[off + n] : -1) : n;
            if (n < N && no >= 0) {
                const int gi = off + no;
                const float rnn = __ldg(&rn[no]);
                // the column's constants: once for the warp's points of one query, else per point
                float ub = 0.f, th = 0.f, c1 = 0.f, c2 = 0.f;
                if (oneq) {
                    ub = __ldg(&Q.ub32[gi]);
                    th = __ldg(&Q.thr[gi]);
                    if (l < L) {
                        c1 = __ldg(&Q.c1[gi]);
                        c2 = __ldg(&Q.c2[gi]);
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (!((vmask >> i) & 1u)) continue;
                    if (!oneq) {
                        const QueryView& Qi = qs[qi[i]];
                        ub = __ldg(&Qi.ub32[gi]);
                        th = __ldg(&Qi.thr[gi]);
                        if (l < L) {
                            c1 = __ldg(&Qi.c1[gi]);
                            c2 = __ldg(&Qi.c2[gi]);
                        }
                    }
                    const float du = (e & 1) ? acc[i][t][e >> 1].y : acc[i][t][e >> 1].x;
                    const float u = ub + du;
                    // |du - exact| <= ||W_i|| (gamma N + E) (a priori), plus the column's threshold
                    const float bound = __fadd_ru(__fmul_ru(rnn, X[i]), th);
                    const bool cert = __fmul_rd(fabsf(u), 1.f - 0x1p-22f) > bound;
                    uncb[i] |= (uint32_t)!cert << slot;
                    flipb[i] |= (uint32_t)(cert && ((u >= 0.f) != (ub >= 0.f))) << slot;
                    if (l < L) {
                        const float dh = act_delta(net.act, du, u, c1, c2);
                        nsum[i] = fmaf(dh, dh, nsum[i]);
                        usum[i] = fmaf(u, u, usum[i]);
                        S.A[mrow[i]][n] = dh;
                    } else {
                        S.A[mrow[i]][n] = u;
                    }
                }
            } else if (n < N || l < L) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if ((vmask >> i) & 1u) S.A[mrow[i]][n] = 0.f;
            }
        }
    }
    if (l < L && HS > HW)  // operand columns past this layer's width: no change
        for (int e = threadIdx.x; e < MT * (HS - HW); e += THREADS)
            S.A[e / (HS - HW)][HW + e % (HS - HW)] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (!((vmask >> i) & 1u)) continue;
        const int m = mrow[i];
        const QueryView& Qi = qs[qi[i]];
        if (uncb[i] && Qi.flip) S.unc[m] = 1;  // signs matter only for coverage
        while (flipb[i]) {
            const int slot = __ffs(flipb[i]) - 1;
            flipb[i] &= flipb[i] - 1u;
            const int np = colb + 32 * (slot >> 2) + (slot & 3);
            const int n = (cmp && l < L) ? Q.perm[off + np] : np;  // neuron
            const int idx = atomicAdd(&S.fcnt[m][l], 1);
            if (idx < FCAP) S.flist[m][l][idx] = (short)n;
            if (Qi.flip) set_bit_once(Qi.flip, off + n);
        }
    }
    // per point: sums over the 8 lanes of its group, then over the NCB column blocks
    // (partials parked in rho, which only an output layer of width <= 32 uses)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float a = nsum[i], b = usum[i], v = chk[i];
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            v = __fadd_ru(v, __shfl_xor_sync(0xffffffffu, v, o));
        }
        if (ng == 0 && ((vmask >> i) & 1u)) {
            float* pp = &S.rho[mrow[i]][3 * cb];
            pp[0] = a;
            pp[1] = b;
            pp[2] = v;
        }
    }
    __syncthreads();  // partials written; every read of the layer's input N, E done
    for (int m = threadIdx.x; m < MT; m += THREADS) {
        if (!S.valid[m]) continue;
        float ns = 0.f, us = 0.f, vc = 0.f;
#pragma unroll
        for (int c = 0; c < NCB; ++c) {
            ns += S.rho[m][3 * c];
            us += S.rho[m][3 * c + 1];
            vc = __fadd_ru(vc, S.rho[m][3 * c + 2]);
        }
        const float Nin = S.N[m], Ein = S.E[m];
        const float vv = __fmul_ru(G, vc);  // ||V||_2^2 bound of the checkpoint sums
        // rounding error vector of the layer, l2: min(a priori, a posteriori)
        const float rpri = __fmul_ru(__fmul_ru(lf, gl), Nin);
        const float rpost = __fmul_ru(lam, __fmul_ru(kUseg, __fmaf_ru(net.frob[l], Nin, __fsqrt_ru(vv))));
        const float rl = fminf(rpri, rpost);
        if (l < L) {
            const float Nl = norm_up(ns);
            // lambda (rounding) + lambda sigma_l E_{l-1} + kvec_l + u N_l
            float El = __fadd_ru(rl, qs[oneq ? 0 : S.q[m]].kvec[l]);
            El = __fmaf_ru(net.lamsig[l], Ein, El);
            El = __fmaf_ru(0x1p-24f, Nl, El);
            if (net.act == ACT_SIGMOID) El = __fmaf_ru(0x1p-26f, norm_up(us), El);
            S.N[m] = Nl;
            S.E[m] = El;
        } else {
            S.N[m] = __fmul_ru(gl, Nin);  // gamma N_{L-1}: a priori dot-product rounding
        }
    }
    __syncthreads();  // N, E and the rows of this layer are final
}

template <int PPW, int NQ, int NQA>
__device__ __forceinline__ void dense_layer(SimtSmem<PPW, NQ>& S, const NetView& net,
                                            const QueryView* __restrict__ qs, int l, int warp,
                                            int lane, bool cmp, bool oneq) {
    // a paired slot width that the blocked layout tiles
    constexpr bool BLK = NQA % 4 == 0 && PPW % 2 == 0 && PPW <= 16 && (NQA * PPW) % 16 == 0 &&
                         NQA * PPW <= 128;
    if constexpr (BLK) {
        dense_blocked<PPW, NQ, (BLK ? NQA : 4)>(S, net, qs, l, warp, lane, cmp, oneq);
        return;
    }
    constexpr int HS = SimtSmem<PPW, NQ>::HS;
    constexpr int HW = 32 * NQA;  // columns of the weight chunk in use
    constexpr bool PER_NEURON = NQA == 1;
    // a narrow layer's weight chunks take more rows of k in the same buffer
    // (fewer chunks, fewer barriers): KCL rows of WSL floats
    constexpr int WSL = HW + 4;
    // (a power of two, so that the chunks tile the operand rows of HS floats)
    constexpr int KFIT = (KC * SimtSmem<PPW, NQ>::WS) / WSL;
    constexpr int KCL = !PER_NEURON ? KC : KFIT >= 64 ? 64 : KFIT >= 32 ? 32 : KFIT >= 16 ? 16 : KC;
    static_assert(2 * KCL * WSL <= 2 * KC * SimtSmem<PPW, NQ>::WS, "weight chunk view exceeds its buffer");
    static_assert(HS % KCL == 0, "weight chunks must tile the operand rows");
    const int L = net.L;
    // compacted (one query whose set-up kept the non-"neg" neurons, see tc.cu):
    // K and N count the kept positions of layers l-1 and l (the output layer keeps
    // its neurons); W_l^T comes from the query's compacted copy, rows of NS floats
    const int NS = net.dims[l];
    const int K = cmp ? qs[0].kc[l - 1] : net.dims[l - 1];
    const int N = (cmp && l < L) ? qs[0].kc[l] : NS;
    const int cntN = (cmp && l < L) ? qs[0].kc[kMaxL + 1 + l] : NS;  // kept neurons
    const float* __restrict__ WT = cmp ? qs[0].wtc[l] : net.WT[l];  // [K][NS]
    const int nchunks = (K + KCL - 1) / KCL;
    // Wide tiles (paired FMAs) read two operand values per shared load and keep
    // the k loop rolled: their accumulators leave no registers for more.
    constexpr bool PAIRED = NQA % 4 == 0;
    constexpr int AK = (PAIRED && PPW * NQA >= 64) ? 2 : 4;
    constexpr int KUNROLL = AK == 2 ? 1 : KCL / AK;
    float* const Wb = &S.Wsm[0][0][0];
    // accumulators in pairs (slots 2i, 2i+1), the operand layout of the paired FMA
    float2 acc[PPW][(NQA + 1) / 2];
    auto accv = [&](int r, int qq) -> float& { return (qq & 1) ? acc[r][qq >> 1].y : acc[r][qq >> 1].x; };
    float chk[PPW];  // PER_NEURON: V_i of this lane's neuron; else sum_g ||s_g||^2 over this lane's neurons
#pragma unroll
    for (int r = 0; r < PPW; ++r) {
        chk[r] = 0.f;
#pragma unroll
        for (int i = 0; i < (NQA + 1) / 2; ++i) acc[r][i] = make_float2(0.f, 0.f);
    }

    const bool vec = (N % 4) == 0 && (NS % 4) == 0;
    auto load_chunk = [&](int c, int buf) {
        float* const dst = Wb + buf * (KCL * WSL);
        if (vec) {
            for (int e = threadIdx.x; e < KCL * (HW / 4); e += THREADS) {
                const int kk = e / (HW / 4), n = (e % (HW / 4)) * 4, k = c * KCL + kk;
                const bool ok = k < K && n < N;
                cp_async16(dst + kk * WSL + n, ok ? (const void*)&WT[(size_t)k * NS + n] : (const void*)WT, ok);
            }
        } else {
            for (int e = threadIdx.x; e < KCL * HW; e += THREADS) {
                const int kk = e / HW, n = e % HW, k = c * KCL + kk;
                const bool ok = k < K && n < N;
                cp_async4(dst + kk * WSL + n, ok ? (const void*)&WT[(size_t)k * NS + n] : (const void*)WT, ok);
            }
        }
        cp_async_commit();
    };
    // A narrow output layer (one neuron per lane, at most 16 outputs): GS lane
    // groups share each output, group g taking the blocks of 4 k whose index is
    // g mod GS; each group sum keeps its own checkpoints (segments of 16 of its
    // terms), and the groups are added after the loop with |each addition's
    // result| added to V (its rounding is at most u times that), so the a
    // posteriori bound u' 16 (V + ||W_i|| ||x||) and the a priori one still hold.
    const int GS = (PER_NEURON && l == L && N >= 1 && N <= 16) ? min(32 / N, 8) : 1;
    const int gq = lane / (N >= 1 ? N : 1), nq = lane - gq * (N >= 1 ? N : 1);
    if (PER_NEURON && GS > 1) {
        // its weights (K x N floats, read by every tile) are loaded straight from
        // global memory and stay in L1: no chunk barriers. The operand rows are
        // this warp's own points (written before the layer's call).
        __syncwarp();
        if (gq < GS) {
            int own = 0;  // this lane's terms so far
            // unrolled so that the loads of several blocks are in flight (each
            // group's sum still runs in order of its k)
#pragma unroll 4
            for (int kb = 4 * gq; kb < K; kb += 4 * GS) {
                if (own > 0 && (own & 15) == 0) {  // checkpoint: this group's partial sums
#pragma unroll
                    for (int r = 0; r < PPW; ++r) chk[r] = __fadd_ru(chk[r], fabsf(acc[r][0].x));
                }
                float4 a4[PPW];
#pragma unroll
                for (int r = 0; r < PPW; ++r) a4[r] = *reinterpret_cast<const float4*>(&S.A[warp * PPW + r][kb]);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k = kb + e;
                    const float w = k < K ? __ldg(&WT[(size_t)k * NS + nq]) : 0.f;
#pragma unroll
                    for (int r = 0; r < PPW; ++r) {
                        const float av = e == 0 ? a4[r].x : e == 1 ? a4[r].y : e == 2 ? a4[r].z : a4[r].w;
                        acc[r][0].x = fmaf(av, w, acc[r][0].x);
                    }
                }
                own += 4;
            }
        }
    } else {
        __syncthreads();  // previous users of Wsm are done
        load_chunk(0, 0);
        for (int c = 0; c < nchunks; ++c) {
            const int buf = c & 1;
            cp_async_wait0();
            __syncthreads();  // chunk c visible to all; chunk c-1's buffer free
            if (c + 1 < nchunks) load_chunk(c + 1, buf ^ 1);
            const float* const wc = Wb + buf * (KCL * WSL);
#pragma unroll KUNROLL
            for (int kk = 0; kk < KCL; kk += AK) {
                const int k0 = c * KCL + kk;
                if (k0 > 0 && k0 % (CKC * KC) == 0) {  // checkpoint: the partial sums at k = k0
#pragma unroll
                    for (int r = 0; r < PPW; ++r) {
                        if (PER_NEURON) {
                            chk[r] = __fadd_ru(chk[r], fabsf(acc[r][0].x));
                        } else {
#pragma unroll
                            for (int qq = 0; qq < NQA; ++qq) chk[r] = __fmaf_ru(accv(r, qq), accv(r, qq), chk[r]);
                        }
                    }
                }
                float av[PPW][AK];
#pragma unroll
                for (int r = 0; r < PPW; ++r) {
                    if (AK == 4) {
                        const float4 t = *reinterpret_cast<const float4*>(&S.A[warp * PPW + r][k0]);
                        av[r][0] = t.x;
                        av[r][1] = t.y;
                        av[r][AK > 2 ? 2 : 0] = t.z;
                        av[r][AK > 3 ? 3 : 0] = t.w;
                    } else {
                        const float2 t = *reinterpret_cast<const float2*>(&S.A[warp * PPW + r][k0]);
                        av[r][0] = t.x;
                        av[r][1] = t.y;
                    }
                }
#pragma unroll
                for (int k4 = 0; k4 < AK; ++k4) {
                    if (PAIRED) {
                        // paired FMA (each half rounds to nearest like fmaf, half the
                        // instructions), one float4 of weights at a time
                        float2 aa[PPW];
#pragma unroll
                        for (int r = 0; r < PPW; ++r) aa[r] = make_float2(av[r][k4], av[r][k4]);
#pragma unroll
                        for (int g = 0; g < NQA / 4; ++g) {
                            const float4 w4 = *reinterpret_cast<const float4*>(wc + (kk + k4) * WSL + 128 * g + 4 * lane);
#pragma unroll
                            for (int r = 0; r < PPW; ++r) {
                                acc[r][2 * g] = __ffma2_rn(aa[r], make_float2(w4.x, w4.y), acc[r][2 * g]);
                                acc[r][2 * g + 1] = __ffma2_rn(aa[r], make_float2(w4.z, w4.w), acc[r][2 * g + 1]);
                            }
                        }
                    } else {
                        float wv[NQA];
#pragma unroll
                        for (int qq = 0; qq < NQA; ++qq) wv[qq] = wc[(kk + k4) * WSL + lane + 32 * qq];
#pragma unroll
                        for (int r = 0; r < PPW; ++r) {
#pragma unroll
                            for (int qq = 0; qq < NQA; ++qq) accv(r, qq) = fmaf(av[r][k4], wv[qq], accv(r, qq));
                        }
                    }
                }
            }
        }
    }

    if (PER_NEURON && GS > 1) {  // add the groups' sums into the lanes of group 0
#pragma unroll
        for (int r = 0; r < PPW; ++r) {
            const float v = acc[r][0].x, vc = chk[r];
            float tot = v, vs = vc;
            for (int g = 1; g < GS; ++g) {
                const float o = __shfl_sync(0xffffffffu, v, (lane + g * N) & 31);
                const float oc = __shfl_sync(0xffffffffu, vc, (lane + g * N) & 31);
                tot = __fadd_rn(tot, o);
                vs = __fadd_ru(vs, __fadd_ru(oc, fabsf(tot)));
            }
            if (gq == 0) {
                acc[r][0].x = tot;
                chk[r] = vs;
            }
        }
    }
    // epilogue of layer l
    const float* rn = net.rownorm[l];
    const int off = net.noff[l];
    const float lf = net.lamfrob[l], gl = net.gam[l];
    const float lam = net.act == ACT_SIGMOID ? 0.25f : 1.0f;
    const float G = (float)((nchunks * KCL + CKC * KC - 1) / (CKC * KC));  // checkpoint segments
    // One query for the warp's points (and a layer wider than a warp): slots
    // outside, points inside, so that each column constant is loaded once for
    // the PPW points; the same operations per point as the loop below.
    const bool one = oneq && !PER_NEURON;
    float nsumA[PPW], usumA[PPW];
    uint32_t uncbA[PPW], flipbA[PPW];
    if (one) {
        const QueryView& Q = qs[0];
        unsigned vmask = 0u;
        float X[PPW];
#pragma unroll
        for (int r = 0; r < PPW; ++r) {
            const int m = warp * PPW + r;
            vmask |= (unsigned)(S.valid[m] != 0) << r;
            X[r] = __fmaf_ru(gl, S.N[m], S.E[m]);
            nsumA[r] = usumA[r] = 0.f;
            uncbA[r] = flipbA[r] = 0u;
        }
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq) {
            const int n = qq < NQA ? slot_neuron<NQA>(lane, qq) : lane + 32 * qq;  // position
            const int no = (cmp && l < L) ? (n < cntN ? Q.perm[off + n] : -1) : n;
            if (qq < NQA && n < N && no >= 0) {
                const int gi = off + no;
                const float ub = __ldg(&Q.ub32[gi]), rnn = __ldg(&rn[no]), th = __ldg(&Q.thr[gi]);
                float c1 = 0.f, c2 = 0.f;
                if (l < L) {
                    c1 = __ldg(&Q.c1[gi]);
                    c2 = __ldg(&Q.c2[gi]);
                }
#pragma unroll
                for (int r = 0; r < PPW; ++r) {
                    if (!((vmask >> r) & 1u)) continue;
                    const int m = warp * PPW + r;
                    const float du = accv(r, qq < NQA ? qq : 0);
                    const float u = ub + du;
                    const float bound = __fadd_ru(__fmul_ru(rnn, X[r]), th);
                    const bool cert = __fmul_rd(fabsf(u), 1.f - 0x1p-22f) > bound;
                    uncbA[r] |= (uint32_t)!cert << qq;
                    flipbA[r] |= (uint32_t)(cert && ((u >= 0.f) != (ub >= 0.f))) << qq;
                    if (l < L) {
                        const float dh = act_delta(net.act, du, u, c1, c2);
                        nsumA[r] = fmaf(dh, dh, nsumA[r]);
                        usumA[r] = fmaf(u, u, usumA[r]);
                        S.A[m][n] = dh;
                    } else {
                        S.A[m][n] = u;
                    }
                }
            } else if ((qq < NQA && n < N) || (l < L && n < HS)) {
#pragma unroll
                for (int r = 0; r < PPW; ++r)
                    if ((vmask >> r) & 1u) S.A[warp * PPW + r][n] = 0.f;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < PPW; ++r) {
        const int m = warp * PPW + r;
        if (!S.valid[m]) continue;
        const QueryView& Q = qs[S.q[m]];
        const float Nin = S.N[m], Ein = S.E[m];
        const float X = __fmaf_ru(gl, Nin, Ein);
        float nsum = 0.f, usum = 0.f;
        uint32_t uncb = 0u, flipb = 0u;  // per slot: uncertain sign, certain change (handled after)
        if (one) {
            nsum = nsumA[r];
            usum = usumA[r];
            uncb = uncbA[r];
            flipb = flipbA[r];
        }
        if (!one) {
#pragma unroll
            for (int qq = 0; qq < NQ; ++qq) {
                const int n = qq < NQA ? slot_neuron<NQA>(lane, qq) : lane + 32 * qq;  // position
                // neuron at position n; -1: a padding position (output change 0)
                const int no = (cmp && l < L) ? (n < cntN ? Q.perm[off + n] : -1) : n;
                if (qq < NQA && n < N && no < 0) {
                    S.A[m][n] = 0.f;
                } else if (qq < NQA && n < N) {
                    const int gi = off + no;
                    const float du = accv(r, qq < NQA ? qq : 0);
                    const float ub = __ldg(&Q.ub32[gi]);
                    const float u = ub + du;
                    const float rnn = __ldg(&rn[no]);
                    // |du - exact|: rounding (a priori, or a posteriori with one neuron per lane) + propagated
                    float bnd = __fmul_ru(rnn, X);
                    if (PER_NEURON) {
                        const float rho = __fmul_ru(kUseg, __fmaf_ru(rnn, Nin, chk[r]));
                        bnd = fminf(bnd, __fmaf_ru(rnn, Ein, rho));
                        if (l == L && no < 32) S.rho[m][no] = fminf(__fmul_ru(rnn, __fmul_ru(gl, Nin)), rho);
                    }
                    const float bound = __fadd_ru(bnd, __ldg(&Q.thr[gi]));
                    const bool cert = __fmul_rd(fabsf(u), 1.f - 0x1p-22f) > bound;
                    uncb |= (uint32_t)!cert << qq;
                    flipb |= (uint32_t)(cert && ((u >= 0.f) != (ub >= 0.f))) << qq;
                    if (l < L) {
                        const float dh = act_delta(net.act, du, u, __ldg(&Q.c1[gi]), __ldg(&Q.c2[gi]));
                        nsum = fmaf(dh, dh, nsum);
                        usum = fmaf(u, u, usum);
                        S.A[m][n] = dh;
                    } else {
                        S.A[m][n] = u;
                    }
                } else if (l < L && n < HS) {
                    S.A[m][n] = 0.f;
                }
            }
        }
        if (uncb && Q.flip) S.unc[m] = 1;  // signs matter only for coverage
        while (flipb) {
            const int qq = __ffs(flipb) - 1;
            flipb &= flipb - 1u;
            const int np = qq < NQA ? slot_neuron<NQA>(lane, qq) : lane + 32 * qq;
            const int n = (cmp && l < L) ? Q.perm[off + np] : np;  // neuron
            const int idx = atomicAdd(&S.fcnt[m][l], 1);
            if (idx < FCAP) S.flist[m][l][idx] = (short)n;
            if (Q.flip) set_bit_once(Q.flip, off + n);
        }
        nsum = warp_sum(nsum);
        usum = warp_sum(usum);
        // ||V||_2 bound of this point's checkpoint sums
        const float vv = PER_NEURON ? warp_sum_ru(__fmul_ru(chk[r], chk[r])) : __fmul_ru(G, warp_sum_ru(chk[r]));
        if (lane == 0) {
            // rounding error vector of the layer, l2: min(a priori, a posteriori)
            const float rpri = __fmul_ru(__fmul_ru(lf, gl), Nin);
            const float rpost = __fmul_ru(lam, __fmul_ru(kUseg, __fmaf_ru(net.frob[l], Nin, __fsqrt_ru(vv))));
            const float rl = fminf(rpri, rpost);
            if (l < L) {
                const float Nl = norm_up(nsum);
                // lambda (rounding) + lambda sigma_l E_{l-1} + kvec_l + u N_l
                float El = __fadd_ru(rl, Q.kvec[l]);
                El = __fmaf_ru(net.lamsig[l], Ein, El);
                El = __fmaf_ru(0x1p-24f, Nl, El);
                if (net.act == ACT_SIGMOID) El = __fmaf_ru(0x1p-26f, norm_up(usum), El);
                S.N[m] = Nl;
                S.E[m] = El;
            } else {
                S.N[m] = __fmul_ru(gl, Nin);  // gamma N_{L-1}: a priori dot-product rounding
            }
        }
    }
    __syncwarp();
}

// Layer 1 of a warp's PPW points when they all belong to one query: the same
// arithmetic as the per-point loop of the kernel (per point, the sum over p in
// order of fl(W_1[j][pix_p] * fl(dv_p / 255))), with each weight and column
// constant loaded once for the PPW points instead of once per point.
template <int PPW, int NQ>
__device__ __forceinline__ void layer1_one_query(SimtSmem<PPW, NQ>& S, const NetView& net,
                                                 const QueryView& Q, int warp, int lane, bool cmp) {
    const int L = net.L, H1 = net.dims[1];
    const int W1 = cmp ? Q.kc[1] : H1;            // positions computed
    const int cnt1 = cmp ? Q.kc[kMaxL + 2] : H1;  // kept neurons
    const int s = Q.s;
    unsigned vmask = 0u;  // valid points of the warp
#pragma unroll
    for (int r = 0; r < PPW; ++r) vmask |= (unsigned)(S.valid[warp * PPW + r] != 0) << r;
    float dus[PPW][NQ];
#pragma unroll
    for (int r = 0; r < PPW; ++r)
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq) dus[r][qq] = 0.f;
    const float* __restrict__ W1T = net.WT[1];  // [H_0][H_1]
    for (int p = 0; p < s; ++p) {
        const float* wr = cmp ? Q.w1c + (size_t)p * H1 : W1T + (size_t)Q.pix[p] * H1;
        float c[PPW];
#pragma unroll
        for (int r = 0; r < PPW; ++r) c[r] = ((vmask >> r) & 1u) ? S.cpx[warp * PPW + r][p] : 0.f;
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq) {
            const int j = lane + 32 * qq;
            if (j < W1) {
                const float w = __ldg(&wr[j]);
#pragma unroll
                for (int r = 0; r < PPW; ++r) dus[r][qq] += __fmul_rn(w, c[r]);
            }
        }
    }
    float nsum[PPW];
    uint32_t uncb[PPW], flipb[PPW];
#pragma unroll
    for (int r = 0; r < PPW; ++r) {
        nsum[r] = 0.f;
        uncb[r] = flipb[r] = 0u;
    }
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) {
        const int j = lane + 32 * qq;                          // position
        const int jo = cmp ? (j < cnt1 ? Q.perm[j] : -1) : j;  // neuron (-1: padding)
        if (j < W1 && jo >= 0) {
            const float ub = __ldg(&Q.ub32[jo]), th = __ldg(&Q.thr[jo]);
            const float c1 = __ldg(&Q.c1[jo]), c2 = __ldg(&Q.c2[jo]);
#pragma unroll
            for (int r = 0; r < PPW; ++r) {
                const float du = dus[r][qq];
                const float u = ub + du;
                const bool cert = __fmul_rd(fabsf(u), 1.f - 0x1p-22f) > th;
                uncb[r] |= (uint32_t)!cert << qq;
                flipb[r] |= (uint32_t)(cert && ((u >= 0.f) != (ub >= 0.f))) << qq;
                const float dh = L > 1 ? act_delta(net.act, du, u, c1, c2) : u;
                nsum[r] = fmaf(dh, dh, nsum[r]);
                S.A[warp * PPW + r][j] = dh;
            }
        } else {
#pragma unroll
            for (int r = 0; r < PPW; ++r) S.A[warp * PPW + r][j] = 0.f;
        }
    }
#pragma unroll
    for (int r = 0; r < PPW; ++r) {
        if (!((vmask >> r) & 1u)) continue;
        const int m = warp * PPW + r;
        if (uncb[r] && Q.flip) S.unc[m] = 1;  // signs matter only for coverage
        while (flipb[r]) {
            const int jp = lane + 32 * (__ffs(flipb[r]) - 1);
            const int j = cmp ? Q.perm[jp] : jp;
            flipb[r] &= flipb[r] - 1u;
            const int idx = atomicAdd(&S.fcnt[m][1], 1);
            if (idx < FCAP) S.flist[m][1][idx] = (short)j;
            if (Q.flip) set_bit_once(Q.flip, j);
        }
        const float ns = warp_sum(nsum[r]);
        if (lane == 0) {
            const float N = norm_up(ns);
            S.N[m] = N;
            S.E[m] = __fmaf_ru(0x1p-24f, N, Q.kvec[1]);
        }
    }
}

// Tiles of at most 64 accumulators per thread are built for two CTAs per SM.
// ONEQ: every tile belongs to query 0 (nq == 1); the instantiation keeps only
// the paths of that case (the other one's code would crowd the instruction cache).
template <int PPW, int NQ, bool ONEQ>
__global__ void __launch_bounds__(THREADS, PPW * NQ <= 64 ? 2 : 1)
k_screen_simt(NetView net, const QueryView* __restrict__ qs, int nq,
              const unsigned long long* __restrict__ tile_prefix, unsigned long long n_tiles,
              const QEntry* __restrict__ gather, const unsigned long long* __restrict__ gather_count,
              unsigned long long gather_cap, Queue out, int out_level, unsigned long long* claim) {
    using Sm = SimtSmem<PPW, NQ>;
    constexpr int MT = Sm::MT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sm& S = *reinterpret_cast<Sm*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = net.L;

    if (ONEQ) nq = 1;
    // compacted columns: one query whose set-up built them (tensor-screen calls)
    const bool cmp = ONEQ && qs[0].compact;
    unsigned long long tiles = n_tiles;
    unsigned long long gcount = 0;
    if (gather) {
        gcount = *gather_count;
        if (gcount > gather_cap) gcount = gather_cap;
        tiles = (gcount + MT - 1) / MT;
    }

    // range mode with a claim counter: tiles in order under the time budget
    unsigned long long* const ctr = gather ? nullptr : claim;
    const unsigned long long deadline =
        (!gather && qs[0].budget_ns) ? qs[0].cnt->t0 + qs[0].budget_ns : 0ull;
    for (unsigned long long ti = 0;; ++ti) {
        if (threadIdx.x == 0) S.g = claim_tile(ctr, ti, tiles, deadline);
        __syncthreads();
        const unsigned long long g = S.g;
        __syncthreads();  // every thread has read S.g before the next claim overwrites it
        if (g == kNoTile) break;
        // ---- S1: decode
        if (lane < PPW) {
            const int m = warp * PPW + lane;
            unsigned long long t = 0;
            int q = 0;
            bool ok;
            if (gather) {
                unsigned long long idx = g * MT + m;
                ok = idx < gcount;
                if (ok) {
                    QEntry e = gather[idx];
                    t = e.t;
                    q = (int)e.q;
                }
            } else {
                int lo = 0, hi = nq - 1;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (tile_prefix[mid] <= g) lo = mid; else hi = mid - 1;
                }
                q = lo;
                const QueryView& Q = qs[q];
                t = (Q.lo & ~31ull) + (g - tile_prefix[q]) * MT + m;
                ok = t >= Q.lo && t < Q.hi;
            }
            S.t[m] = t;
            S.q[m] = q;
            S.valid[m] = ok;
            S.unc[m] = 0;
            S.vstate[m] = 0;
#pragma unroll
            for (int l = 0; l <= kMaxL; ++l) S.fcnt[m][l] = 0;
            if (ok) {
                const QueryView& Q = qs[q];
                int d[kMaxS];
                decode_digits(t, Q.s, Q.R, d);
                for (int p = 0; p < Q.s; ++p) {
                    S.dig[m][p] = (unsigned char)d[p];
                    S.cpx[m][p] = __fdiv_rn((float)Q.dv[p * Q.R + d[p]], 255.f);
                }
                if (!gather && Q.filter && !in_filter(Q, d)) S.valid[m] = 0;  // L2 ball / shell
            }
        }
        __syncwarp();
        if (!gather && lane == 0) {  // points that pass a filter are counted here
            const QueryView& Q = qs[S.q[warp * PPW]];
            if (Q.filter) {
                int c = 0;
                for (int r = 0; r < PPW; ++r) c += S.valid[warp * PPW + r];
                if (c) atomicAdd(&Q.cnt->n_points, (unsigned long long)c);
            }
        }

        // ---- S2/S3: layer 1 from the delta tables
        if (ONEQ) {
            layer1_one_query<PPW, NQ>(S, net, qs[0], warp, lane, cmp);
            __syncwarp();
        } else {
            const int H1 = net.dims[1];
            const int W1 = cmp ? qs[0].kc[1] : H1;               // positions computed
            const int cnt1 = cmp ? qs[0].kc[kMaxL + 2] : H1;     // kept neurons
            for (int r = 0; r < PPW; ++r) {
                const int m = warp * PPW + r;
                if (!S.valid[m]) continue;
                const QueryView& Q = qs[S.q[m]];
                const int s = Q.s;
                // du_j = sum_p fl(W_1[j][pix_p] * fl(dv_p / 255)), p in order (Eq. 1 on the
                // s changed pixels): the s weight rows of the query's pixels are shared by
                // all points and stay in L1. Per term at most 2u |t_p| from the exact
                // product, plus the FP32 sum: inside the table-sum bound e1 of the prologue.
                float dus[NQ];
#pragma unroll
                for (int qq = 0; qq < NQ; ++qq) dus[qq] = 0.f;
                const float* __restrict__ W1T = net.WT[1];  // [H_0][H_1]
                for (int p = 0; p < s; ++p) {
                    // validated by the prologue; compacted: the query's row of W_1 weights
                    const float* wr = cmp ? Q.w1c + (size_t)p * H1 : W1T + (size_t)Q.pix[p] * H1;
                    const float c = S.cpx[m][p];
#pragma unroll
                    for (int qq = 0; qq < NQ; ++qq) {
                        const int j = lane + 32 * qq;
                        if (j < W1) dus[qq] += __fmul_rn(__ldg(&wr[j]), c);
                    }
                }
                // branch-free over the slots (their loads pipeline); uncertain signs
                // and certain changes are collected as bits and handled after
                float nsum = 0.f;
                uint32_t uncb = 0u, flipb = 0u;
#pragma unroll
                for (int qq = 0; qq < NQ; ++qq) {
                    const int j = lane + 32 * qq;                       // position
                    const int jo = cmp ? (j < cnt1 ? Q.perm[j] : -1) : j;  // neuron (-1: padding)
                    float dh = 0.f;
                    if (j < W1 && jo >= 0) {
                        const float du = dus[qq];
                        const float ub = __ldg(&Q.ub32[jo]);
                        const float u = ub + du;
                        const bool cert = __fmul_rd(fabsf(u), 1.f - 0x1p-22f) > __ldg(&Q.thr[jo]);
                        uncb |= (uint32_t)!cert << qq;
                        flipb |= (uint32_t)(cert && ((u >= 0.f) != (ub >= 0.f))) << qq;
                        if (L > 1) dh = act_delta(net.act, du, u, __ldg(&Q.c1[jo]), __ldg(&Q.c2[jo]));
                        else dh = u;
                        nsum = fmaf(dh, dh, nsum);
                    }
                    S.A[m][j] = dh;
                }
                if (uncb && Q.flip) S.unc[m] = 1;  // signs matter only for coverage
                while (flipb) {
                    const int jp = lane + 32 * (__ffs(flipb) - 1);
                    const int j = cmp ? Q.perm[jp] : jp;
                    flipb &= flipb - 1u;
                    const int idx = atomicAdd(&S.fcnt[m][1], 1);
                    if (idx < FCAP) S.flist[m][1][idx] = (short)j;
                    if (Q.flip) set_bit_once(Q.flip, j);
                }
                nsum = warp_sum(nsum);
                if (lane == 0) {
                    const float N = norm_up(nsum);
                    S.N[m] = N;
                    S.E[m] = __fmaf_ru(0x1p-24f, N, Q.kvec[1]);
                }
            }
            __syncwarp();
        }

        // ---- S4: dense layers on the deltas
        for (int l = 2; l <= L; ++l) {
            if (net.dims[l] <= 32) {
                dense_layer<PPW, NQ, 1>(S, net, qs, l, warp, lane, cmp, ONEQ);
                continue;
            }
            // a compacted hidden layer narrower than the variant's width runs with
            // fewer slots per lane (whole 128-column groups: the paired slot layout)
            const int ng = (cmp && l < L) ? (qs[0].kc[l] + 127) / 128 : NQ;
            if (NQ % 8 == 0 && NQ >= 8 && 8 * ng <= NQ)
                dense_layer<PPW, NQ, (NQ % 8 == 0 && NQ >= 8 ? NQ / 2 : NQ)>(S, net, qs, l, warp, lane, cmp, ONEQ);
            else if (NQ % 16 == 0 && 16 * ng <= 3 * NQ)
                dense_layer<PPW, NQ, (NQ % 16 == 0 ? 3 * NQ / 4 : NQ)>(S, net, qs, l, warp, lane, cmp, ONEQ);
            else
                dense_layer<PPW, NQ, NQ>(S, net, qs, l, warp, lane, cmp, ONEQ);
        }

        // ---- S5: verdict (layer L values are in A[m][0..H_L))
        {
            const int HL = net.dims[L], offL = net.noff[L];
            const float* rn = net.rownorm[L];
            for (int r = 0; r < PPW; ++r) {
                const int m = warp * PPW + r;
                if (!S.valid[m]) continue;
                const QueryView& Q = qs[S.q[m]];
                const int D = Q.cnt->D;
                // per output: rounding rho_o (a priori ||W_o|| gamma N, or the a posteriori
                // bound of the output layer); shared error ||W_D - W_o|| E
                const float gN = L > 1 ? S.N[m] : 0.f;
                const float Ep = L > 1 ? S.E[m] : 0.f;
                auto rho = [&](int o) { return L == 1 ? 0.f : HL <= 32 ? S.rho[m][o] : __fmul_ru(rn[o], gN); };
                const float yD = S.A[m][D];
                const float rhD = rho(D);
                const float dD = Q.dub[offL + D];
                if (Q.prop == PROP_THRESHOLD) {  // Eq. 11: per output rho_o + ||W_o|| E + dub_o
                    const float V = (float)Q.V;
                    bool da = false, db = false, oa = false, ob = true;
                    for (int o = lane; o < HL; o += 32) {
                        const float ro = L > 1 ? rn[o] : 0.f;
                        const float e = __fmaf_ru(ro, Ep, __fadd_ru(rho(o), __fadd_ru(Q.dub[offL + o],
                                                                                      (float)(2.0 * kTau))));
                        const int sd = thr_side(S.A[m][o], V, e);
                        if (o == D) { da = sd > 0; db = sd < 0; }
                        else { oa = oa || sd > 0; ob = ob && sd < 0; }
                    }
                    da = __any_sync(0xffffffffu, da);
                    db = __any_sync(0xffffffffu, db);
                    oa = __any_sync(0xffffffffu, oa);
                    ob = __all_sync(0xffffffffu, ob);
                    if (lane == 0) S.vstate[m] = thr_verdict(da, db, oa, ob);
                    continue;
                }
                bool unsafe = false, safe = true;
                for (int o = lane; o < HL; o += 32) {
                    if (o == D) continue;
                    const float yo = S.A[m][o];
                    const float diff = yD - yo;
                    const float pw = L > 1 ? net.pairw[D * HL + o] : 0.f;
                    float eb = __fadd_ru(__fadd_ru(rhD, rho(o)),
                                         __fadd_ru(__fadd_ru(dD, Q.dub[offL + o]), (float)(2.0 * kTau)));
                    eb = __fmaf_ru(pw, Ep, eb);
                    eb = __fmaf_ru(0x1p-23f, __fadd_ru(__fadd_ru(fabsf(yD), fabsf(yo)), fabsf(diff)), eb);
                    if (diff < -eb) unsafe = true;
                    else if (!(diff > eb)) safe = false;
                }
                unsafe = __any_sync(0xffffffffu, unsafe);
                safe = __all_sync(0xffffffffu, safe);
                if (lane == 0) S.vstate[m] = unsafe ? 1 : (safe ? 0 : 2);
            }
            __syncwarp();
        }

        // ---- S6/S7: per-point results (lane r < PPW holds point warp*PPW + r)
        {
            const int m = warp * PPW + (lane < PPW ? lane : 0);
            const bool mine = lane < PPW && S.valid[m];
            const QueryView& Q = qs[S.q[m]];
            bool bad = mine && (S.unc[m] || S.vstate[m] == 2);
            if (mine && !bad && Q.ss)
                for (int l = 1; l < L; ++l)
                    if (S.fcnt[m][l] == 1 && S.fcnt[m][l + 1] > FCAP) bad = true;
            queue_push_warp(out, bad, S.t[m], (unsigned)S.q[m], Q.cnt, out_level);
            const bool adv = mine && !bad && S.vstate[m] == 1;
            // the warp's points are consecutive indices of one query in range mode
            const unsigned am = __ballot_sync(0xffffffffu, adv);
            if (am) {
                if (!gather) {
                    if (lane == __ffs(am) - 1) {
                        atomicAdd(&Q.cnt->n_adv, (unsigned long long)__popc(am));
                        atomicMin(&Q.cnt->first, S.t[m]);
                    }
                    if (adv && Q.bitmap && S.t[m] < Q.bitmap_bits) set_bit_atomic(Q.bitmap, S.t[m]);
                } else if (adv) {
                    record_adversarial(Q, S.t[m]);
                }
            }
            if (mine && !bad && Q.ss) {
                for (int l = 1; l < L; ++l) {
                    if (S.fcnt[m][l] != 1) continue;
                    const int j = S.flist[m][l][0];
                    const int Hn = net.dims[l + 1];
                    const int nt = S.fcnt[m][l + 1];
                    for (int e = 0; e < nt; ++e)
                        set_bit_once(Q.ss, (unsigned long long)net.ssoff[l] +
                                               (unsigned long long)j * Hn + S.flist[m][l + 1][e]);
                }
            }
        }
        __syncwarp();
        if (gather) {  // time to verdict: this warp's queued points are resolved
            const int m = warp * PPW + (lane < PPW ? lane : 0);
            const bool mine = lane < PPW && S.valid[m];
            const unsigned vm = __ballot_sync(0xffffffffu, mine);
            if (mine) {
                const unsigned peers = __match_any_sync(vm, S.q[m]);
                if (lane == __ffs(peers) - 1) work_done(qs[S.q[m]].cnt, __popc(peers));
            }
        } else {  // time to verdict: one screen tile of the query is done
            __syncthreads();
            if (threadIdx.x == 0) work_done(qs[S.q[0]].cnt, 1);
        }
    }
}

template <int PPW, int NQ>
void launch_variant(const NetView& net, const QueryView* d_qs, int nq, const unsigned long long* tp,
                    unsigned long long n_tiles, const QEntry* gather, const unsigned long long* gc,
                    unsigned long long gcap, Queue out, int level, int n_sm, cudaStream_t st,
                    unsigned long long* claim = nullptr) {
    const size_t smem = sizeof(SimtSmem<PPW, NQ>);
    auto kern = nq == 1 ? k_screen_simt<PPW, NQ, true> : k_screen_simt<PPW, NQ, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = smem < 60000 ? 2 : 1;
    const int tuned = gather ? net.simt_ctas_gather : net.simt_ctas_range;
    if (tuned >= 1 && tuned <= 8) per_sm = tuned;
    unsigned long long grid = (unsigned long long)n_sm * per_sm;
    if (!gather && n_tiles < grid) grid = n_tiles ? n_tiles : 1;
    kern<<<(unsigned)grid, THREADS, smem, st>>>(net, d_qs, nq, tp, n_tiles, gather, gc, gcap, out,
                                                level, claim);
}

}  // namespace simt
}  // namespace vbmc
