// wide.cu -- tensor-core screen for wide ReLU nets: hidden layers of up to 1024
// neurons on tcgen05 (E4M3 with kind::f8f6f4, BF16/FP16 with kind::f16), one
// layer per launch over a chunk of points, with a proven error bound per point.
//
// For each chunk of consecutive points of the index space:
//   k_wide_l1     one warp per point: layer 1 from the delta tables (Eq. 1), the
//                 ReLU in delta form dh_1 = relu(ub + du) - relu(ub), certain
//                 sign changes, and the rounded operand of layer 2 (E4M3: with
//                 the point's scale s = max_j |dh_1,j| / 448)
//   k_wide_gemm   per hidden layer l >= 2: du_l = What_l dh_{l-1} as 128-point x
//                 256-neuron tiles (TMA-fed operand ring, double-buffered TMEM
//                 accumulators), fused epilogue: scales, certain signs against
//                 the point's bound, delta ReLU, the rounded operand of layer
//                 l+1, sums of squares of dh_l and of its rounding residual
//   k_wide_stats  per point: N_l, R_l, E_l of dh_l
//   k_wide_out    one thread per point: output layer in FP32 from the rounded
//                 operand, margin and class (Eq. 10) or the threshold literal
//                 (Eq. 11), output signs, SS-Cover
//                 (Sec. III-B); undecided points go to the recheck queue
// then the chunk's undecided points run through the FP32, double-float and FP64
// passes.
//
// Operands: dh^ = s round(dh / s), the values the MMA multiplies (s = 1 for
// 16-bit types); R = ||dh - dh^|| is computed from the values. Error of du_l,n
// (a_n = ||What_n||, b_n = ||W_n - What_n||, N = ||dh_{l-1}||, E = bound on the
// error of dh_{l-1}, u_acc = K x the accumulation unit of wide.h):
//   |err| <= a_n (R + E + u_acc (N + R)) + b_n (N + E) + 2^-22 |du_n|
// and the layer's error vector propagates with spectral-norm bounds.
// Signs only matter for coverage: with coverage off no point is rechecked
// because a sign was uncertain (value errors are in the bound either way).
#include "dev.cuh"
#include "launch.h"
#include "tc_ptx.cuh"
#include "wide.h"
#include "tc.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace vbmc {

namespace {

constexpr int W_STAGES = 3;
constexpr int W_THREADS = 320;   // producer warp, MMA warp, 8 epilogue warps
constexpr int W_BM = 128;        // points per tile (MMA M)
constexpr int W_BN = 256;        // neurons per tile (MMA N)
constexpr int W_BKB = 128;       // bytes per K chunk (one 128-byte swizzle row)
constexpr unsigned long long W_CHUNK = 1ull << 20;
constexpr float kE4M3Max = 448.f;

template <int ET>
struct Elem;
template <>
struct Elem<WIDE_E4M3> {
    static constexpr int bytes = 1;
    __device__ static uint32_t round(float x, float& back) {
        const __nv_fp8_e4m3 q(x);
        back = static_cast<float>(q);
        return (uint32_t)q.__x;
    }
    __device__ static float value(uint32_t bits) {
        __nv_fp8_e4m3 q;
        q.__x = (__nv_fp8_storage_t)bits;
        return static_cast<float>(q);
    }
};
template <>
struct Elem<WIDE_BF16> {
    static constexpr int bytes = 2;
    __device__ static uint32_t round(float x, float& back) {
        const __nv_bfloat16 q = __float2bfloat16_rn(x);
        back = __bfloat162float(q);
        return (uint32_t)__bfloat16_as_ushort(q);
    }
    __device__ static float value(uint32_t bits) { return __bfloat162float(__ushort_as_bfloat16((unsigned short)bits)); }
};
template <>
struct Elem<WIDE_FP16> {
    static constexpr int bytes = 2;
    __device__ static uint32_t round(float x, float& back) {
        const __half q = __float2half_rn(x);
        back = __half2float(q);
        return (uint32_t)__half_as_ushort(q);
    }
    __device__ static float value(uint32_t bits) { return __half2float(__ushort_as_half((unsigned short)bits)); }
};

struct WSmem {
    uint8_t A[W_STAGES][W_BM * W_BKB];
    uint8_t B[W_STAGES][W_BN * W_BKB];
    unsigned long long bars[2 * W_STAGES + 5];
    uint32_t tmem_slot;
    int abort_flag;
};

__device__ __forceinline__ int FULL(int i) { return i; }
__device__ __forceinline__ int EMPTY(int i) { return W_STAGES + i; }
constexpr int ACCF0 = 2 * W_STAGES;  // accumulator buffer ready (2)
constexpr int ACCE0 = ACCF0 + 2;     // accumulator buffer drained (2)
constexpr int FINB = ACCF0 + 4;

__device__ __forceinline__ float norm_up(float s) { return __fsqrt_ru(__fmul_ru(s, 1.0002f)); }

// Per-point state inside the chunk workspace.
struct WDev {
    float *scale, *n2, *r2, *sN, *sR, *sE;
    unsigned char* unc;
    int* fcnt;
    short* flist;
    unsigned long long chunk;
    int row_bytes;
};

__device__ __forceinline__ void record_flip(const WDev& w, int l, unsigned long long i, int neuron) {
    const int k = atomicAdd(&w.fcnt[(size_t)l * w.chunk + i], 1);
    if (k < kWideFcap) w.flist[((size_t)l * w.chunk + i) * kWideFcap + k] = (short)neuron;
}

// Pack the rounded bits of element e (of a lane's run) into 32-bit words.
template <int ET>
__device__ __forceinline__ void pack(uint32_t* words, int e, uint32_t bits) {
    if (Elem<ET>::bytes == 1) words[e >> 2] |= bits << (8 * (e & 3));
    else words[e >> 1] |= bits << (16 * (e & 1));
}

// ------------------------------------------------------------------ layer 1

template <int ET>
__global__ void __launch_bounds__(256) k_wide_l1(NetView net, const QueryView* qs, unsigned long long lo,
                                                 unsigned long long count, uint8_t* A_out, WDev w) {
    constexpr int EB = Elem<ET>::bytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long i = (unsigned long long)blockIdx.x * 8 + warp;
    if (i >= count) return;
    const QueryView& Q = qs[0];
    const bool cov = Q.flip != nullptr;
    const int H1 = net.dims[1];
    const int per = H1 >> 5;  // 8..32 columns per lane, a multiple of 8
    const int j0 = lane * per;
    int d[kMaxS];
    decode_digits(lo + i, Q.s, Q.R, d);
    if (Q.filter && !in_filter(Q, d)) {  // outside the L2 ball / shell: a zero row, skipped later
        uint32_t* row = reinterpret_cast<uint32_t*>(A_out + i * (unsigned long long)w.row_bytes);
        for (int k = lane; k < w.row_bytes / 4; k += 32) row[k] = 0u;
        if (lane == 0) {
            const size_t at = (size_t)1 * w.chunk + i;
            w.scale[at] = 1.f;
            w.sN[at] = w.sR[at] = w.sE[at] = 0.f;
            w.unc[i] = 2;
        }
        return;
    }
    if (Q.filter && lane == 0) atomicAdd(&Q.cnt->n_points, 1ull);  // points that pass are counted
    float du[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) du[e] = 0.f;
    for (int p = 0; p < Q.s; ++p) {
        const float4* row = reinterpret_cast<const float4*>(Q.tab + ((size_t)p * Q.R + d[p]) * H1 + j0);
#pragma unroll
        for (int e4 = 0; e4 < 8; ++e4) {
            if (4 * e4 >= per) break;
            const float4 v = __ldg(row + e4);
            du[4 * e4] += v.x;
            du[4 * e4 + 1] += v.y;
            du[4 * e4 + 2] += v.z;
            du[4 * e4 + 3] += v.w;
        }
    }
    bool unc = false;
    float dh[32], m = 0.f;
#pragma unroll
    for (int e = 0; e < 32; ++e) {
        if (e >= per) break;
        const int j = j0 + e;
        const float ub = Q.ub32[j];
        const float u = ub + du[e];
        if (cov) {
            if (!(__fmul_rd(fabsf(u), 1.f - 0x1p-22f) > Q.thr[j])) unc = true;
            else if ((u >= 0.f) != (ub >= 0.f)) {
                record_flip(w, 1, i, j);
                set_bit_once(Q.flip, (unsigned long long)j);
            }
        }
        dh[e] = fmaxf(du[e] + Q.c1[j], Q.c2[j]);
        m = fmaxf(m, fabsf(dh[e]));
    }
    float s = 1.f;
    if (ET == WIDE_E4M3) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        s = m > 0.f ? m / kE4M3Max : 1.f;
    }
    const float inv = 1.f / s;
    float ns = 0.f, rs = 0.f;
    uint32_t words[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) words[k] = 0u;
#pragma unroll
    for (int e = 0; e < 32; ++e) {
        if (e >= per) break;
        float back;
        const uint32_t b = Elem<ET>::round(dh[e] * inv, back);
        const float r = dh[e] - s * back;
        ns = fmaf(dh[e], dh[e], ns);
        rs = fmaf(r, r, rs);
        pack<ET>(words, e, b);
    }
    uint32_t* dst = reinterpret_cast<uint32_t*>(A_out + i * (unsigned long long)w.row_bytes + (size_t)j0 * EB);
    const int nw = per * EB / 4;
#pragma unroll
    for (int k = 0; k < 16; ++k)
        if (k < nw) dst[k] = words[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ns += __shfl_xor_sync(0xffffffffu, ns, o);
        rs += __shfl_xor_sync(0xffffffffu, rs, o);
    }
    const bool any_unc = __any_sync(0xffffffffu, unc);
    if (lane == 0) {
        const float N = norm_up(ns);
        const size_t at = (size_t)1 * w.chunk + i;
        w.scale[at] = s;
        w.sN[at] = N;
        w.sR[at] = __fmaf_ru(0x1p-22f, N, norm_up(rs));
        w.sE[at] = __fmaf_ru(0x1p-24f, N, Q.kvec[1]);
        if (any_unc) w.unc[i] = 1;
    }
}

// ------------------------------------------------------------------ hidden GEMM

struct WGemmArgs {
    CUtensorMap ta;  // operand of layer l: [chunk][K]
    CUtensorMap tb;  // Wq_l [N][K]
    int l, K, N;
    unsigned long long count;
    const float* sw;
    const float* a;
    const float* b;
    float sq;        // bound of sigma(What): E4M3 scale of the next operand
    float acc_unit;  // accumulation error per product
    uint8_t* A_out;
    unsigned int* err;
};

template <int ET>
__global__ void __launch_bounds__(W_THREADS, 1)
k_wide_gemm(const __grid_constant__ WGemmArgs G, NetView net, const QueryView* qs, WDev w) {
    constexpr int EB = Elem<ET>::bytes;
    constexpr int KE = W_BKB / EB;  // elements per K chunk
    extern __shared__ uint8_t smem_raw[];
    WSmem& S = *reinterpret_cast<WSmem*>(smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* abortp = &S.abort_flag;
    const int nb = G.N / W_BN, kch = G.K / KE;
    const unsigned long long mb = (G.count + W_BM - 1) / W_BM;
    const unsigned long long ntiles = mb * (unsigned long long)nb;
    auto bar = [&](int i) { return tc::smem_u32(&S.bars[i]); };
    if (threadIdx.x == 0) {
        for (int i = 0; i < W_STAGES; ++i) {
            tc::mbar_init(bar(FULL(i)), 1);
            tc::mbar_init(bar(EMPTY(i)), 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(bar(ACCF0 + i), 1);
            tc::mbar_init(bar(ACCE0 + i), 8);
        }
        tc::mbar_init(bar(FINB), 1);
        S.abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tc::smem_u32(&S.tmem_slot), 512);
        tc::tmem_relinquish();
    }
    if (warp == 0 && lane == 0) {
        tc::prefetch_tmap(&G.ta);
        tc::prefetch_tmap(&G.tb);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = S.tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (unsigned long long g = blockIdx.x; g < ntiles && ok; g += gridDim.x) {
                const int m = (int)(g / nb), n = (int)(g % nb);
                for (int kc = 0; kc < kch; ++kc) {
                    const int slot = it % W_STAGES;
                    if (!tc::mbar_wait(bar(EMPTY(slot)), ((it / W_STAGES) & 1) ^ 1, abortp)) {
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(bar(FULL(slot)), (uint32_t)(W_BM + W_BN) * W_BKB);
                    tc::tma_load_2d(tc::smem_u32(S.A[slot]), &G.ta, kc * KE, m * W_BM, bar(FULL(slot)));
                    tc::tma_load_2d(tc::smem_u32(S.B[slot]), &G.tb, kc * KE, n * W_BN, bar(FULL(slot)));
                    ++it;
                }
            }
            if (!ok) {  // let the copies already issued land before the CTA leaves
                const uint64_t t0 = tc::global_ns();
                for (uint32_t i = it > (uint32_t)W_STAGES ? it - W_STAGES : 0; i < it; ++i)
                    while (!tc::mbar_try(bar(FULL(i % W_STAGES)), (i / W_STAGES) & 1) &&
                           tc::global_ns() - t0 < tc::kWaitNs) {
                    }
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            uint32_t it = 0, tl = 0;
            bool ok = true;
            const uint32_t idesc = ET == WIDE_E4M3 ? tc::idesc_e4m3(W_BM, W_BN)
                                                   : tc::idesc_f16(W_BM, W_BN, ET == WIDE_BF16);
            for (unsigned long long g = blockIdx.x; g < ntiles && ok; g += gridDim.x, ++tl) {
                const uint32_t buf = tl & 1;
                if (!tc::mbar_wait(bar(ACCE0 + buf), ((tl >> 1) & 1) ^ 1, abortp)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t d = tmem + buf * W_BN;
                for (int kc = 0; kc < kch; ++kc) {
                    const int slot = it % W_STAGES;
                    if (!tc::mbar_wait(bar(FULL(slot)), (it / W_STAGES) & 1, abortp)) { ok = false; break; }
                    tc::tc_fence_after();
                    const uint32_t a0 = tc::smem_u32(S.A[slot]), b0 = tc::smem_u32(S.B[slot]);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t ad = tc::desc_sw128(a0 + ks * 32), bd = tc::desc_sw128(b0 + ks * 32);
                        if (ET == WIDE_E4M3) tc::mma_f8(d, ad, bd, idesc, (kc | ks) != 0);
                        else tc::mma_f16(d, ad, bd, idesc, (kc | ks) != 0);
                    }
                    tc::mma_commit(bar(EMPTY(slot)));
                    ++it;
                }
                if (ok) tc::mma_commit(bar(ACCF0 + buf));
            }
            tc::mma_commit(bar(FINB));
            const uint64_t t0 = tc::global_ns();
            while (!tc::mbar_try(bar(FINB), 0) && tc::global_ns() - t0 < tc::kWaitNs) {
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const QueryView& Q = qs[0];
        const bool cov = Q.flip != nullptr;
        const int qd = warp & 3, hf = (warp - 2) >> 2;
        const int l = G.l;
        const int off = net.noff[l];
        const float uacc = (float)G.K * G.acc_unit;
        uint32_t tl = 0;
        for (unsigned long long g = blockIdx.x; g < ntiles; g += gridDim.x, ++tl) {
            if (*abortp) break;
            const uint32_t buf = tl & 1;
            const int m = (int)(g / nb), n = (int)(g % nb);
            const unsigned long long i = (unsigned long long)m * W_BM + 32 * qd + lane;
            const bool valid = i < G.count && w.unc[i] != 2;  // 2: outside the query's filter
            float sin = 0.f, Nn = 0.f, Rr = 0.f, Ee = 0.f;
            if (valid) {
                const size_t at = (size_t)(l - 1) * w.chunk + i;
                sin = w.scale[at];
                Nn = w.sN[at];
                Rr = w.sR[at];
                Ee = w.sE[at];
            }
            const float Pa = __fmaf_ru(uacc, __fadd_ru(Nn, Rr), __fadd_ru(Rr, Ee));
            const float Pb = __fadd_ru(Nn, Ee);
            float sout = 1.f;
            if (ET == WIDE_E4M3) {
                const float big = __fmul_ru(G.sq, __fadd_ru(__fadd_ru(Nn, Rr), Ee)) * (1.f + 0x1p-6f);
                sout = big > 0.f ? big / kE4M3Max : 1.f;
            }
            const float inv = 1.f / sout;
            if (!tc::mbar_wait(bar(ACCF0 + buf), (tl >> 1) & 1, abortp)) break;
            tc::tc_fence_after();
            bool unc = false;
            float ns = 0.f, rs = 0.f;
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const int col0 = n * W_BN + hf * 128 + 32 * c;
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + buf * W_BN + (uint32_t)(hf * 128 + 32 * c), v);
                uint32_t words[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) words[k] = 0u;
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    const int col = col0 + e, gi = off + col;
                    const float du = __fmul_rn(__fmul_rn(v[e], sin), __ldg(&G.sw[col]));
                    if (valid && cov) {
                        const float ub = __ldg(&Q.ub32[gi]);
                        const float u = ub + du;
                        float bound =
                            __fmaf_ru(__ldg(&G.a[col]), Pa, __fmaf_ru(__ldg(&G.b[col]), Pb, __ldg(&Q.thr[gi])));
                        bound = __fmaf_ru(0x1p-22f, fabsf(du), bound);
                        if (!(__fmul_rd(fabsf(u), 1.f - 0x1p-22f) > bound)) unc = true;
                        else if ((u >= 0.f) != (ub >= 0.f)) {
                            record_flip(w, l, i, col);
                            set_bit_once(Q.flip, (unsigned long long)gi);
                        }
                    }
                    const float dh = fmaxf(du + __ldg(&Q.c1[gi]), __ldg(&Q.c2[gi]));
                    float back;
                    const uint32_t bq = Elem<ET>::round(dh * inv, back);
                    const float r = dh - sout * back;
                    ns = fmaf(dh, dh, ns);
                    rs = fmaf(r, r, rs);
                    pack<ET>(words, e, bq);
                }
                if (valid) {
                    uint4* dst = reinterpret_cast<uint4*>(G.A_out + i * (unsigned long long)w.row_bytes +
                                                          (size_t)col0 * EB);
#pragma unroll
                    for (int k = 0; k < 2 * EB; ++k)
                        dst[k] = make_uint4(words[4 * k], words[4 * k + 1], words[4 * k + 2], words[4 * k + 3]);
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(bar(ACCE0 + buf));
            if (valid) {
                const size_t at = (size_t)l * w.chunk + i;
                atomicAdd(&w.n2[at], ns);
                atomicAdd(&w.r2[at], rs);
                if (unc) w.unc[i] = 1;
                if (n == 0 && hf == 0) w.scale[at] = sout;
            }
        }
    }
    // ---- teardown: every issued tensor-core op has completed (FIN) before TMEM goes back
    tc::tc_fence_before();
    __syncthreads();
    if (*abortp && threadIdx.x == 0) atomicOr(G.err, DERR_TC_WAIT);
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

// N_l, R_l, E_l of dh_l for every point of the chunk (after layer l's GEMM).
__global__ void k_wide_stats(WDev w, unsigned long long count, int l, float sq, float sd, float fq, float uacc,
                             const QueryView* qs) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const size_t p = (size_t)(l - 1) * w.chunk + i, at = (size_t)l * w.chunk + i;
    const float Np = w.sN[p], Rp = w.sR[p], Ep = w.sE[p];
    const float N = norm_up(w.n2[at]);
    // ||err(du_l)|| <= sq R + sd N + (sq + sd) E + u_acc ||What||_F (N + R), plus the
    // FP32 rounding of the epilogue (2^-21 (sq + sd)(N + E)) and of dh_l (2^-24 N_l)
    float El = __fmul_ru(sq, Rp);
    El = __fmaf_ru(sd, Np, El);
    El = __fmaf_ru(__fadd_ru(sq, sd), Ep, El);
    El = __fmaf_ru(__fmul_ru(uacc, fq), __fadd_ru(Np, Rp), El);
    El = __fmaf_ru(__fmul_ru(0x1p-21f, __fadd_ru(sq, sd)), __fadd_ru(Np, Ep), El);
    El = __fadd_ru(El, qs[0].kvec[l]);
    El = __fmaf_ru(0x1p-24f, N, El);
    w.sN[at] = N;
    w.sR[at] = __fmaf_ru(0x1p-22f, N, norm_up(w.r2[at]));
    w.sE[at] = El;
}

// ------------------------------------------------------------------ output layer

template <int ET>
__global__ void __launch_bounds__(256) k_wide_out(NetView net, const QueryView* qs, unsigned long long lo,
                                                  unsigned long long count, const uint8_t* A_in, WDev w,
                                                  Queue out, int out_level) {
    constexpr int EB = Elem<ET>::bytes;
    constexpr int PER16 = 16 / EB;  // elements per 16-byte load
    extern __shared__ float Ws[];   // [H_L][K]
    const int L = net.L, K = net.dims[L - 1], HL = net.dims[L];
    for (int e = threadIdx.x; e < HL * K; e += blockDim.x) Ws[e] = net.W[L][e];
    __syncthreads();
    const QueryView& Q = qs[0];
    const bool cov = Q.flip != nullptr;
    const int D = Q.cnt->D, offL = net.noff[L];
    const float gam = (float)(K + 2) * 0x1p-24f;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        float acc[kWideOut];
#pragma unroll
        for (int o = 0; o < kWideOut; ++o) acc[o] = 0.f;
        const size_t at = (size_t)(L - 1) * w.chunk + i;
        const float s = w.scale[at], Nn = w.sN[at], Rr = w.sR[at], Ee = w.sE[at];
        const uint4* row = reinterpret_cast<const uint4*>(A_in + i * (unsigned long long)w.row_bytes);
        for (int jc = 0; jc < K / PER16; ++jc) {
            const uint4 q4 = row[jc];
            const uint32_t qw[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
            for (int b = 0; b < PER16; ++b) {
                const uint32_t bits = EB == 1 ? (qw[b >> 2] >> (8 * (b & 3))) & 0xFFu
                                              : (qw[b >> 1] >> (16 * (b & 1))) & 0xFFFFu;
                const float x = s * Elem<ET>::value(bits);
                const int j = jc * PER16 + b;
#pragma unroll
                for (int o = 0; o < kWideOut; ++o)
                    if (o < HL) acc[o] = fmaf(Ws[o * K + j], x, acc[o]);
            }
        }
        const unsigned long long t = lo + i;
        if (w.unc[i] == 2) continue;  // outside the query's filter
        bool bad = w.unc[i] != 0;
        float y[kWideOut];
        float yD = 0.f;
        const float RE = __fadd_ru(Rr, Ee), NR = __fadd_ru(Nn, Rr);
#pragma unroll
        for (int o = 0; o < kWideOut; ++o) {
            y[o] = 0.f;
            if (o >= HL) continue;
            const float ub = Q.ub32[offL + o];
            const float u = ub + acc[o];
            y[o] = u;
            if (o == D) yD = u;
            if (!cov) continue;  // output signs matter only for coverage
            const float wn = net.rownorm[L][o];
            const float bound = __fmaf_ru(wn, RE, __fmaf_ru(__fmul_ru(gam, wn), NR, Q.thr[offL + o]));
            if (!(__fmul_rd(fabsf(u), 1.f - 0x1p-22f) > bound)) bad = true;
            else if ((u >= 0.f) != (ub >= 0.f)) {
                record_flip(w, L, i, o);
                set_bit_once(Q.flip, (unsigned long long)(offL + o));
            }
        }
        bool unsafe = false, safe = true;
        const float dD = Q.dub[offL + D];
        if (Q.prop == PROP_THRESHOLD) {  // Eq. 11: per output ||W_o|| (R + E + gamma (N + R)) + dub_o
            const float V = (float)Q.V;
            bool da = false, db = false, oa = false, ob = true;
#pragma unroll
            for (int o = 0; o < kWideOut; ++o) {
                if (o >= HL) continue;
                const float wn = net.rownorm[L][o];
                const float e = __fmaf_ru(wn, RE, __fmaf_ru(__fmul_ru(gam, wn), NR,
                                                            __fadd_ru(Q.dub[offL + o], (float)(2.0 * kTau))));
                const int sd = thr_side(y[o], V, e);
                if (o == D) { da = sd > 0; db = sd < 0; }
                else { oa = oa || sd > 0; ob = ob && sd < 0; }
            }
            const int vv = thr_verdict(da, db, oa, ob);
            unsafe = vv == 1;
            safe = vv == 0;
        }
#pragma unroll
        for (int o = 0; o < kWideOut; ++o) {
            if (Q.prop == PROP_THRESHOLD || o >= HL || o == D) continue;
            const float diff = yD - y[o];
            float eb = __fmul_ru(net.pairw[D * HL + o], RE);
            eb = __fmaf_ru(__fmul_ru(gam, __fadd_ru(net.rownorm[L][D], net.rownorm[L][o])), NR, eb);
            eb = __fadd_ru(eb, __fadd_ru(__fadd_ru(dD, Q.dub[offL + o]), (float)(2.0 * kTau)));
            eb = __fmaf_ru(0x1p-23f, __fadd_ru(__fadd_ru(fabsf(yD), fabsf(y[o])), fabsf(diff)), eb);
            if (diff < -eb) unsafe = true;
            else if (!(diff > eb)) safe = false;
        }
        if (!unsafe && !safe) bad = true;
        if (!bad && Q.ss)
            for (int l = 1; l < L; ++l)
                if (w.fcnt[(size_t)l * w.chunk + i] == 1 && w.fcnt[(size_t)(l + 1) * w.chunk + i] > kWideFcap)
                    bad = true;
        if (bad) {
            queue_push(out, t, 0u, Q.cnt, out_level);
        } else {
            if (unsafe) record_adversarial(Q, t);
            if (Q.ss)
                for (int l = 1; l < L; ++l) {
                    if (w.fcnt[(size_t)l * w.chunk + i] != 1) continue;
                    const int j = w.flist[((size_t)l * w.chunk + i) * kWideFcap];
                    const int Hn = net.dims[l + 1];
                    const int nt = w.fcnt[(size_t)(l + 1) * w.chunk + i];
                    for (int e = 0; e < nt; ++e)
                        set_bit_once(Q.ss, (unsigned long long)net.ssoff[l] + (unsigned long long)j * Hn +
                                               w.flist[((size_t)(l + 1) * w.chunk + i) * kWideFcap + e]);
                }
        }
    }
}

__global__ void k_wide_work_done(const QueryView* qs) { work_done(qs[0].cnt, 1); }

// Diagnostic copy of the operand rows of dh_m (m = 1..L-1) for points 0..n-1.
template <int ET>
__global__ void k_wide_trace(const uint8_t* A, WDev w, int m, int H, WideTrace t) {
    constexpr int EB = Elem<ET>::bytes;
    const int i = blockIdx.x;
    if (i >= t.n) return;
    const size_t at = (size_t)m * w.chunk + i;
    const float sc = w.scale[at];
    const uint8_t* row = A + (size_t)i * w.row_bytes;
    float* out = t.vals + ((size_t)(m - 1) * t.n + i) * t.hmax;
    for (int j = threadIdx.x; j < H; j += blockDim.x) {
        const uint32_t bits = EB == 1 ? (uint32_t)row[j] : (uint32_t)reinterpret_cast<const uint16_t*>(row)[j];
        out[j] = Elem<ET>::value(bits) * sc;
    }
    if (threadIdx.x == 0) {
        float* o = t.nre + ((size_t)(m - 1) * t.n + i) * 3;
        o[0] = w.sN[at];
        o[1] = w.sR[at];
        o[2] = w.sE[at];
    }
}

const WideTrace* g_trace = nullptr;

// ------------------------------------------------------------------ E4M3 self-test

// One 128 x 256 x 128 E4M3 product through the same TMA, descriptor and MMA path.
__global__ void __launch_bounds__(128, 1)
k_wide_selftest(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, float* out,
                int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t* sa = base;
    uint8_t* sb = base + W_BM * W_BKB;
    __shared__ unsigned long long bars[2];
    __shared__ uint32_t slot;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        tc::mbar_init(tc::smem_u32(&bars[0]), 1);
        tc::mbar_init(tc::smem_u32(&bars[1]), 1);
        abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&slot), 256);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = slot;
    bool ok = true;
    if (threadIdx.x == 0) {
        tc::mbar_expect_tx(tc::smem_u32(&bars[0]), (uint32_t)(W_BM + W_BN) * W_BKB);
        tc::tma_load_2d(tc::smem_u32(sa), &ta, 0, 0, tc::smem_u32(&bars[0]));
        tc::tma_load_2d(tc::smem_u32(sb), &tb, 0, 0, tc::smem_u32(&bars[0]));
        ok = tc::mbar_wait(tc::smem_u32(&bars[0]), 0, &abort_flag);
        if (ok) {
            tc::tc_fence_after();
            const uint32_t idesc = tc::idesc_e4m3(W_BM, W_BN);
            for (int ks = 0; ks < 4; ++ks)
                tc::mma_f8(tmem, tc::desc_sw128(tc::smem_u32(sa) + ks * 32), tc::desc_sw128(tc::smem_u32(sb) + ks * 32),
                           idesc, ks != 0);
        }
        tc::mma_commit(tc::smem_u32(&bars[1]));
        if (!tc::mbar_wait(tc::smem_u32(&bars[1]), 0, &abort_flag)) ok = false;
        if (!ok) atomicExch(status, 2);
    }
    __syncthreads();
    tc::tc_fence_after();
    if (!abort_flag) {
        for (int c = 0; c < W_BN; c += 32) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
            for (int e = 0; e < 32; ++e) out[(size_t)(32 * warp + lane) * W_BN + c + e] = v[e];
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 256);
    }
}

// ------------------------------------------------------------------ host helpers

float up_f(double x) {
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, INFINITY);
    return f;
}

// E4M3 (bias 7, 3 mantissa bits, no infinities, max 448) of a float, round to
// nearest even, saturating: the byte and its value.
uint8_t e4m3_byte(float x, double* val) {
    const double ax = std::fabs((double)x);
    const uint8_t sign = x < 0.f ? 0x80 : 0x00;
    if (!(ax > 0.0)) {
        *val = 0.0;
        return 0;
    }
    if (ax >= 448.0) {
        *val = x < 0 ? -448.0 : 448.0;
        return sign | 0x7E;
    }
    int e = (int)std::floor(std::log2(ax));
    if (e < -6) e = -6;  // subnormal range: spacing 2^-9
    const double step = std::ldexp(1.0, e - 3);
    double q = std::nearbyint(ax / step) * step;  // ties to even (default rounding mode)
    if (q >= 448.0) q = 448.0;
    uint8_t code;
    if (q < std::ldexp(1.0, -6)) {
        code = (uint8_t)std::lrint(q / std::ldexp(1.0, -9));  // subnormal: 0.mmm x 2^-6
    } else {
        int ee = (int)std::floor(std::log2(q));
        const double mant = q / std::ldexp(1.0, ee) - 1.0;  // in [0, 1)
        const int mbits = (int)std::lrint(mant * 8.0);
        if (mbits == 8) {
            ++ee;
            code = (uint8_t)(((ee + 7) << 3));
        } else {
            code = (uint8_t)(((ee + 7) << 3) | mbits);
        }
    }
    *val = x < 0.f ? -q : q;
    return sign | code;
}

// 16-bit rounding of a float on the host (round to nearest even), bits and value.
uint16_t bf16_bits(float x, double* val) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    const uint16_t b = (uint16_t)(u >> 16);
    uint32_t back = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &back, 4);
    *val = f;
    return b;
}

uint16_t fp16_bits(float x, double* val) {
    const __half h = __float2half_rn(x);
    *val = (double)__half2float(h);
    return __half_as_ushort(h);
}

bool encode_map(PFN_cuTensorMapEncodeTiled_v12000 encode, CUtensorMap* m, int type, const void* ptr,
                unsigned long long inner_elems, unsigned long long rows, unsigned long long stride_bytes,
                unsigned box_rows) {
    const int eb = type == WIDE_E4M3 ? 1 : 2;
    const CUtensorMapDataType dt = type == WIDE_E4M3   ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                   : type == WIDE_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                       : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    cuuint64_t gdim[2] = {(cuuint64_t)inner_elems, (cuuint64_t)rows};
    cuuint64_t gstr[1] = {(cuuint64_t)stride_bytes};
    cuuint32_t box[2] = {(cuuint32_t)(W_BKB / eb), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return encode(m, dt, 2, const_cast<void*>(ptr), gdim, gstr, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&encode, 12000, cudaEnableDefault,
                                         &qr) != cudaSuccess)
        return nullptr;
    return encode;
}

// The E4M3 self-test: small integer operands (exact products and sums in any
// accumulator of 12 or more bits), plus probe rows 125..127 of A and 253..255 of
// B whose dot products need 18 to 23 significand bits (exact in FP32).
// *fp32_acc = 1 when every probe sum came back exact.
vbmc_status selftest_e4m3(PFN_cuTensorMapEncodeTiled_v12000 encode, int* fp32_acc) {
    std::vector<uint8_t> ha((size_t)W_BM * W_BKB), hb((size_t)W_BN * W_BKB);
    std::vector<double> va(ha.size()), vb(hb.size());
    for (size_t e = 0; e < ha.size(); ++e) ha[e] = e4m3_byte((float)((int)((e * 7 + 3) % 5) - 2), &va[e]);
    for (size_t e = 0; e < hb.size(); ++e) hb[e] = e4m3_byte((float)((int)((e * 11 + 1) % 5) - 2), &vb[e]);
    auto set_row = [](std::vector<uint8_t>& h, std::vector<double>& v, int row, float first, float rest) {
        for (int k = 0; k < W_BKB; ++k)
            h[(size_t)row * W_BKB + k] = e4m3_byte(k == 0 ? first : rest, &v[(size_t)row * W_BKB + k]);
    };
    set_row(ha, va, 127, 448.f, 0x1p-9f);  // 448 + 127 x 2^-9 (with B row 255)
    set_row(ha, va, 126, 448.f, 0x1p-6f);  // 448 + 127 x 2^-12 (with B row 254)
    set_row(ha, va, 125, 256.f, 0x1p-9f);  // 256 + 127 x 2^-15 (with B row 253)
    set_row(hb, vb, 255, 1.f, 1.f);
    set_row(hb, vb, 254, 1.f, 0x1p-6f);
    set_row(hb, vb, 253, 1.f, 0x1p-6f);
    uint8_t *da = nullptr, *db = nullptr;
    float* dout = nullptr;
    int* dst = nullptr;
    vbmc_status res = VBMC_ERR_CUDA;
    CUtensorMap ta, tb;
    std::vector<float> got((size_t)W_BM * W_BN);
    int status = 0;
    if (cudaMalloc(&da, ha.size()) != cudaSuccess || cudaMalloc(&db, hb.size()) != cudaSuccess ||
        cudaMalloc(&dout, sizeof(float) * got.size()) != cudaSuccess || cudaMalloc(&dst, sizeof(int)) != cudaSuccess)
        goto done;
    cudaMemcpy(da, ha.data(), ha.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(db, hb.data(), hb.size(), cudaMemcpyHostToDevice);
    cudaMemset(dst, 0, sizeof(int));
    if (!encode_map(encode, &ta, WIDE_E4M3, da, W_BKB, W_BM, W_BKB, W_BM) ||
        !encode_map(encode, &tb, WIDE_E4M3, db, W_BKB, W_BN, W_BKB, W_BN))
        goto done;
    {
        const size_t smem = (size_t)(W_BM + W_BN) * W_BKB + 1024;
        cudaFuncSetAttribute(k_wide_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_wide_selftest<<<1, 128, smem>>>(ta, tb, dout, dst);
        if (cudaDeviceSynchronize() != cudaSuccess) goto done;
        cudaMemcpy(got.data(), dout, sizeof(float) * got.size(), cudaMemcpyDeviceToHost);
        cudaMemcpy(&status, dst, sizeof(int), cudaMemcpyDeviceToHost);
        if (status != 0) goto done;
        res = VBMC_OK;
        *fp32_acc = 1;
        for (int r = 0; r < W_BM && res == VBMC_OK; ++r)
            for (int n = 0; n < W_BN; ++n) {
                double ex = 0.0;
                for (int k = 0; k < W_BKB; ++k) ex += va[(size_t)r * W_BKB + k] * vb[(size_t)n * W_BKB + k];
                if ((double)got[(size_t)r * W_BN + n] == ex) continue;
                if (r >= 125 || n >= 253) {
                    *fp32_acc = 0;  // a probe sum lost bits: short accumulator
                } else {
                    res = VBMC_ERR_UNSUPPORTED;  // wrong products or layout
                    break;
                }
            }
    }
done:
    cudaFree(da);
    cudaFree(db);
    cudaFree(dout);
    cudaFree(dst);
    return res;
}

template <int ET>
void launch_chunk(const WidePrec& P, int type, WideWork& w, const WDev& dv, const NetView& v, QueryView* d_q,
                  unsigned long long c0, unsigned long long count, unsigned int* err, Queue q32, int n_sm,
                  cudaStream_t st, const WideTrace* trace) {
    const int L = v.L;
    const size_t gemm_smem = sizeof(WSmem) + 1024;
    cudaFuncSetAttribute(k_wide_gemm<ET>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem);
    const size_t out_smem = sizeof(float) * (size_t)v.dims[L] * v.dims[L - 1];
    cudaFuncSetAttribute(k_wide_out<ET>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out_smem);
    k_wide_l1<ET><<<(unsigned)((count + 7) / 8), 256, 0, st>>>(v, d_q, c0, count, w.A[0], dv);
    if (trace && count >= (unsigned long long)trace->n)
        k_wide_trace<ET><<<trace->n, 256, 0, st>>>(w.A[0], dv, 1, v.dims[1], *trace);
    for (int l = 2; l < L; ++l) {
        const WideLayer& ly = P.ly[l];
        WGemmArgs G;
        G.ta = w.tA[type][l % 2][l];
        G.tb = ly.tw;
        G.l = l;
        G.K = ly.K;
        G.N = ly.N;
        G.count = count;
        G.sw = ly.sw;
        G.a = ly.a;
        G.b = ly.b;
        G.sq = ly.sq;
        G.acc_unit = P.acc_unit;
        G.A_out = w.A[(l + 1) % 2];
        G.err = err;
        const unsigned long long tiles = ((count + W_BM - 1) / W_BM) * (unsigned long long)(ly.N / W_BN);
        const unsigned grid = (unsigned)std::min<unsigned long long>((unsigned long long)n_sm, tiles);
        k_wide_gemm<ET><<<grid, W_THREADS, gemm_smem, st>>>(G, v, d_q, dv);
        k_wide_stats<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(dv, count, l, ly.sq, ly.sd, ly.fq,
                                                                     (float)ly.K * P.acc_unit, d_q);
        if (trace && count >= (unsigned long long)trace->n)
            k_wide_trace<ET><<<trace->n, 256, 0, st>>>(w.A[(l + 1) % 2], dv, l, ly.N, *trace);
    }
    k_wide_out<ET><<<(unsigned)std::min<unsigned long long>((count + 255) / 256, (unsigned long long)n_sm * 8), 256,
                     out_smem, st>>>(v, d_q, c0, count, w.A[L % 2], dv, q32, 1);
}

}  // namespace

void wide_set_trace(const WideTrace* t) { g_trace = t; }

int wide_type(int precision) {
    if (precision == VBMC_PREC_FP8) return WIDE_E4M3;
    if (precision == VBMC_PREC_BF16) return WIDE_BF16;
    if (precision == VBMC_PREC_FP16) return WIDE_FP16;
    return -1;
}

bool wide_supported(const NetView& v) {
    if (v.act != ACT_RELU || v.L < 2 || v.L > kMaxL) return false;
    for (int l = 1; l < v.L; ++l)
        if (v.dims[l] % 256 || v.dims[l] > 1024) return false;
    if (v.dims[v.L] > kWideOut) return false;
    return true;
}

vbmc_status wide_build(WideNet& wn, const NetView& v, const std::vector<std::vector<float>>& W, int type) {
    if (type < 0 || type >= WIDE_NTYPES) return VBMC_ERR_ARG;
    WidePrec& P = wn.prec[type];
    if (P.ready) return VBMC_OK;
    (void)cudaGetLastError();
    PFN_cuTensorMapEncodeTiled_v12000 encode = get_encode();
    if (!encode) return VBMC_ERR_CUDA;
    if (type == WIDE_E4M3) {
        int fp32_acc = 0;
        const vbmc_status st = selftest_e4m3(encode, &fp32_acc);
        if (st != VBMC_OK) return st;
        P.acc_unit = fp32_acc ? kWideAccFp32 : kWideAccShort;
    } else {
        // BF16 / FP16: the kind::f16 accumulator probe of the fused screen
        float u = 0.f;
        const vbmc_status st = tc_f16_selftest(type == WIDE_BF16, &u, nullptr, nullptr);
        if (st != VBMC_OK) return st;
        P.acc_unit = u;
    }
    const int eb = type == WIDE_E4M3 ? 1 : 2;
    for (int l = 2; l < v.L; ++l) {
        const int K = v.dims[l - 1], N = v.dims[l];
        WideLayer& ly = P.ly[l];
        ly.K = K;
        ly.N = N;
        std::vector<uint8_t> hq((size_t)N * K * eb);
        std::vector<float> sw(N), a(N), b(N);
        std::vector<double> What((size_t)N * K), Wd((size_t)N * K);
        double f2 = 0.0;
        for (int n = 0; n < N; ++n) {
            float s = 1.f;
            if (type == WIDE_E4M3) {
                double mx = 0.0;
                for (int k = 0; k < K; ++k) mx = std::max(mx, std::fabs((double)W[l][(size_t)n * K + k]));
                s = mx > 0.0 ? (float)(mx / 448.0) : 1.f;
            }
            sw[n] = s;
            double a2 = 0.0, b2 = 0.0;
            for (int k = 0; k < K; ++k) {
                const float wv = W[l][(size_t)n * K + k];
                double q;
                const size_t e = (size_t)n * K + k;
                if (type == WIDE_E4M3) {
                    hq[e] = e4m3_byte(wv / s, &q);
                } else {
                    const uint16_t bits = type == WIDE_BF16 ? bf16_bits(wv, &q) : fp16_bits(wv, &q);
                    std::memcpy(&hq[2 * e], &bits, 2);
                }
                const double wh = q * (double)s;
                What[e] = wh;
                Wd[e] = (double)wv - wh;
                a2 += wh * wh;
                b2 += ((double)wv - wh) * ((double)wv - wh);
            }
            f2 += a2;
            a[n] = up_f(std::sqrt(a2) * (1.0 + 1e-9));
            b[n] = up_f(std::sqrt(b2) * (1.0 + 1e-9));
        }
        ly.fq = up_f(std::sqrt(f2) * (1.0 + 1e-9));
        ly.sq = up_f(spectral_bound(What, N, K));
        ly.sd = up_f(spectral_bound(Wd, N, K));
        if (!(ly.sq > 0.f)) return VBMC_ERR_CUDA;
        void* dq = nullptr;
        float *dsw = nullptr, *da = nullptr, *db = nullptr;
        if (cudaMalloc(&dq, hq.size()) != cudaSuccess) return VBMC_ERR_OOM;
        wn.owned.push_back(dq);
        if (cudaMalloc(&dsw, sizeof(float) * N) != cudaSuccess) return VBMC_ERR_OOM;
        wn.owned.push_back(dsw);
        if (cudaMalloc(&da, sizeof(float) * N) != cudaSuccess) return VBMC_ERR_OOM;
        wn.owned.push_back(da);
        if (cudaMalloc(&db, sizeof(float) * N) != cudaSuccess) return VBMC_ERR_OOM;
        wn.owned.push_back(db);
        cudaMemcpy(dq, hq.data(), hq.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(dsw, sw.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
        cudaMemcpy(da, a.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
        cudaMemcpy(db, b.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
        ly.wq = dq;
        ly.sw = dsw;
        ly.a = da;
        ly.b = db;
        if (!encode_map(encode, &ly.tw, type, dq, K, N, (unsigned long long)K * eb, W_BN)) return VBMC_ERR_CUDA;
    }
    if (cudaGetLastError() != cudaSuccess) return VBMC_ERR_CUDA;
    P.ready = true;
    return VBMC_OK;
}

void wide_free(WideNet& wn) {
    for (void* p : wn.owned) cudaFree(p);
    wn.owned.clear();
    for (auto& p : wn.prec) p.ready = false;
}

vbmc_status wide_work_alloc(WideWork& w, const NetView& v, unsigned long long chunk) {
    if (w.chunk) return VBMC_OK;
    if (chunk == 0) chunk = W_CHUNK;
    chunk = (chunk + 127) & ~127ull;
    int kmax = 0;
    for (int l = 1; l < v.L; ++l) kmax = std::max(kmax, v.dims[l]);
    const int row_bytes = 2 * kmax;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(p, bytes ? bytes : 16);
        if (e == cudaSuccess) w.owned.push_back((void*)*p);
    };
    const size_t per_layer = (size_t)(kMaxL + 1) * chunk;
    A(&w.A[0], (size_t)chunk * row_bytes);
    A(&w.A[1], (size_t)chunk * row_bytes);
    A(&w.scale, sizeof(float) * per_layer);
    A(&w.n2, sizeof(float) * per_layer);
    A(&w.r2, sizeof(float) * per_layer);
    A(&w.sN, sizeof(float) * per_layer);
    A(&w.sR, sizeof(float) * per_layer);
    A(&w.sE, sizeof(float) * per_layer);
    A(&w.unc, chunk);
    A(&w.fcnt, sizeof(int) * per_layer);
    A(&w.flist, sizeof(short) * per_layer * kWideFcap);
    if (e != cudaSuccess) {
        wide_work_free(w);
        return VBMC_ERR_OOM;
    }
    PFN_cuTensorMapEncodeTiled_v12000 encode = get_encode();
    if (!encode) {
        wide_work_free(w);
        return VBMC_ERR_CUDA;
    }
    for (int type = 0; type < WIDE_NTYPES; ++type)
        for (int l = 2; l < v.L; ++l)  // the output layer reads its operand with plain loads
            if (!encode_map(encode, &w.tA[type][l % 2][l], type, w.A[l % 2], (unsigned long long)v.dims[l - 1],
                            chunk, (unsigned long long)row_bytes, W_BM)) {
                wide_work_free(w);
                return VBMC_ERR_CUDA;
            }
    w.chunk = chunk;
    w.row_bytes = row_bytes;
    return VBMC_OK;
}

void wide_work_free(WideWork& w) {
    for (void* p : w.owned) cudaFree(p);
    w.owned.clear();
    w.chunk = 0;
}

vbmc_status wide_run(const WideNet& wn, int type, WideWork& w, const NetView& v, QueryView* d_q,
                     unsigned long long lo, unsigned long long hi, unsigned long long* d_qcount,
                     QEntry* const* d_queue, unsigned long long cap, int n_sm, cudaStream_t st) {
    if (type < 0 || type >= WIDE_NTYPES || !wn.prec[type].ready || !w.chunk) return VBMC_ERR_STATE;
    const WDev dv{w.scale, w.n2, w.r2, w.sN, w.sR, w.sE, w.unc, w.fcnt, w.flist, w.chunk, w.row_bytes};
    Queue q32{d_queue[1], d_qcount + 1, cap};
    Queue qdf{d_queue[2], d_qcount + 2, cap};
    Queue q64{d_queue[3], d_qcount + 3, cap};
    // the query's error flags (for waits that gave up) live in its counters
    QueryView hq;
    if (cudaMemcpyAsync(&hq, d_q, sizeof(QueryView), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return VBMC_ERR_CUDA;
    unsigned int* err = &hq.cnt->err;
    for (unsigned long long c0 = lo; c0 < hi; c0 += w.chunk) {
        const unsigned long long count = std::min<unsigned long long>(w.chunk, hi - c0);
        cudaMemsetAsync(d_qcount, 0, sizeof(unsigned long long) * 4, st);
        cudaMemsetAsync(w.n2, 0, sizeof(float) * (size_t)(kMaxL + 1) * w.chunk, st);
        cudaMemsetAsync(w.r2, 0, sizeof(float) * (size_t)(kMaxL + 1) * w.chunk, st);
        cudaMemsetAsync(w.unc, 0, count, st);
        cudaMemsetAsync(w.fcnt, 0, sizeof(int) * (size_t)(kMaxL + 1) * w.chunk, st);
        const WidePrec& P = wn.prec[type];
        const WideTrace* tr = c0 == lo ? g_trace : nullptr;
        if (type == WIDE_E4M3) launch_chunk<WIDE_E4M3>(P, type, w, dv, v, d_q, c0, count, err, q32, n_sm, st, tr);
        else if (type == WIDE_BF16) launch_chunk<WIDE_BF16>(P, type, w, dv, v, d_q, c0, count, err, q32, n_sm, st, tr);
        else launch_chunk<WIDE_FP16>(P, type, w, dv, v, d_q, c0, count, err, q32, n_sm, st, tr);
        // this chunk's undecided points: FP32, double-float, FP64 passes
        launch_screen_simt(v, d_q, 1, nullptr, 0, d_queue[1], d_qcount + 1, cap, qdf, 2, n_sm, st);
        launch_df(v, d_q, 1, d_queue[2], d_qcount + 2, cap, q64, 3, n_sm, st);
        launch_fp64(v, d_q, 1, d_queue[3], d_qcount + 3, cap, 0, 0, n_sm, st);
    }
    k_wide_work_done<<<1, 1, 0, st>>>(d_q);
    return cudaGetLastError() == cudaSuccess ? VBMC_OK : VBMC_ERR_CUDA;
}

}  // namespace vbmc
