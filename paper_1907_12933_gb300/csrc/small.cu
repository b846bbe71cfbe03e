// small.cu -- the FP32 pass for small nets (every layer at most 32 neurons, as
// the paper's 25-x-y classifiers): one thread per point, weights, tables and
// per-neuron constants in shared memory, sign changes gathered in a CTA-local
// mask. Same arithmetic, in the same order, and the same error bound as the
// warp-per-point FP32 pass (screen_simt.cuh):
//   layer 1   du_j = sum_p tab[p][d_p][j] (Eq. 1, incremental), u = ub + du
//   layer l   du = W_l dh_{l-1}, sequential FMA over the inputs
//   bounds    X_l = gamma_{H_{l-1}} N_{l-1} + E_{l-1}, |du_i - exact| <= ||W_l,i|| X_l,
//             E_l = lambda ||W_l||_F gamma N_{l-1} + lambda sigma_l E_{l-1} + kvec_l + 2^-24 N_l
//             (+ 2^-26 ||u_l|| for sigmoid)
//   verdict   margin pairs of Eq. 10 against ||W_D|| + ||W_o|| times gamma N_{L-1}
//             plus ||W_D - W_o|| E_{L-1}
// A point with an uncertain sign (coverage on) or an undecided margin goes on to
// the next pass.
#include "dev.cuh"
#include "launch.h"

#include <cmath>

namespace vbmc {
namespace {

constexpr int SM_THREADS = 256;  // points per tile
constexpr int SM_MAXW = 32;      // widest layer
constexpr int SM_MAXL = 4;       // weight layers
constexpr int SM_FCAP = 6;       // sign changes kept per point and layer
constexpr int SM_TAB = 4096;     // floats of delta tables in shared memory
constexpr int SM_FW = 8;         // flip-mask words (<= 256 neurons)

__device__ __forceinline__ float norm_up_s(float s) { return __fsqrt_ru(__fmul_ru(s, 1.0002f)); }

__device__ __forceinline__ float act_delta_s(int act, float du, float u, float c1, float c2) {
    if (act == ACT_RELU) return fmaxf(du + c1, c2);
    if (act == ACT_SIGMOID) return 1.0f / (1.0f + expf(-u)) - c2;
    return du;
}

struct SmallSmem {
    float tab[SM_TAB];
    float W[SM_MAXL + 1][SM_MAXW * SM_MAXW];  // W[l][i * K + k]
    float rn[SM_MAXL + 1][SM_MAXW];
    float ub32[SM_MAXL * SM_MAXW + 1], thr[SM_MAXL * SM_MAXW + 1], c1[SM_MAXL * SM_MAXW + 1],
        c2[SM_MAXL * SM_MAXW + 1], dub[SM_MAXL * SM_MAXW + 1];
    uint32_t cflip[SM_FW];
};

// One point: returns its state; fills its certain sign changes.
__global__ void __launch_bounds__(SM_THREADS)
k_small(NetView net, const QueryView* __restrict__ qs, const unsigned long long* __restrict__ tile_prefix,
        unsigned long long n_tiles, const QEntry* __restrict__ gather,
        const unsigned long long* __restrict__ gather_count, unsigned long long gather_cap, Queue out,
        int out_level) {
    __shared__ SmallSmem S;
    const QueryView& Q = qs[0];
    const int L = net.L, total = net.total;
    const int SR = Q.s * Q.R * net.dims[1];
    const bool tab_sm = SR <= SM_TAB;  // larger tables are read through the L1 cache
    if (tab_sm)
        for (int e = threadIdx.x; e < SR; e += blockDim.x) S.tab[e] = Q.tab[e];
    for (int l = 2; l <= L; ++l) {
        const int K = net.dims[l - 1], N = net.dims[l];
        for (int e = threadIdx.x; e < K * N; e += blockDim.x) S.W[l][e] = net.W[l][e];
        for (int e = threadIdx.x; e < N; e += blockDim.x) S.rn[l][e] = net.rownorm[l][e];
    }
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        S.ub32[e] = Q.ub32[e];
        S.thr[e] = Q.thr[e];
        S.c1[e] = Q.c1[e];
        S.c2[e] = Q.c2[e];
        S.dub[e] = Q.dub[e];
    }
    if (threadIdx.x < SM_FW) S.cflip[threadIdx.x] = 0u;
    __syncthreads();
    const bool cov = Q.flip != nullptr;
    const int lane = threadIdx.x & 31;
    unsigned long long tiles = n_tiles, gcount = 0;
    if (gather) {
        gcount = *gather_count;
        if (gcount > gather_cap) gcount = gather_cap;
        tiles = (gcount + SM_THREADS - 1) / SM_THREADS;
    }
    const unsigned long long base = Q.lo & ~31ull;
    const int D = Q.cnt->D, HL = net.dims[L], offL = net.noff[L];
    for (unsigned long long g = blockIdx.x; g < tiles; g += gridDim.x) {
        unsigned long long t = 0;
        bool ok;
        if (gather) {
            const unsigned long long idx = g * SM_THREADS + threadIdx.x;
            ok = idx < gcount;
            if (ok) t = gather[idx].t;
        } else {
            t = base + g * SM_THREADS + threadIdx.x;
            ok = t >= Q.lo && t < Q.hi;
        }
        bool unc = false, ssover = false;
        int vstate = 0;
        int fcnt[SM_MAXL + 1];
        short flist[SM_MAXL + 1][SM_FCAP];
#pragma unroll
        for (int l = 0; l <= SM_MAXL; ++l) fcnt[l] = 0;
        int d[kMaxS];
        if (ok) {
            decode_digits(t, Q.s, Q.R, d);
            if (!gather && Q.filter) ok = in_filter(Q, d);  // L2 ball / shell
        }
        if (!gather && Q.filter) {  // points that pass the filter are counted here
            const unsigned vm = __ballot_sync(0xffffffffu, ok);
            if (lane == 0 && vm) atomicAdd(&Q.cnt->n_points, (unsigned long long)__popc(vm));
        }
        if (ok) {
            const int H1 = net.dims[1];
            float h[SM_MAXW];
            float nsum = 0.f;
            for (int j = 0; j < H1; ++j) {
                float du = 0.f;
                for (int p = 0; p < Q.s; ++p) {
                    const int at = (p * Q.R + d[p]) * H1 + j;
                    du += tab_sm ? S.tab[at] : __ldg(&Q.tab[at]);
                }
                const float ub = S.ub32[j];
                const float u = ub + du;
                if (!(__fmul_rd(fabsf(u), 1.f - 0x1p-22f) > S.thr[j])) {
                    if (cov) unc = true;  // signs matter only for coverage
                } else if ((u >= 0.f) != (ub >= 0.f)) {
                    if (fcnt[1] < SM_FCAP) flist[1][fcnt[1]] = (short)j;
                    ++fcnt[1];
                    if (cov) atomicOr(&S.cflip[j >> 5], 1u << (j & 31));
                }
                const float dh = L > 1 ? act_delta_s(net.act, du, u, S.c1[j], S.c2[j]) : u;
                nsum = fmaf(dh, dh, nsum);
                h[j] = dh;
            }
            float Nn = norm_up_s(nsum);
            float Ee = __fmaf_ru(0x1p-24f, Nn, Q.kvec[1]);
            for (int l = 2; l <= L; ++l) {
                const int K = net.dims[l - 1], N = net.dims[l], off = net.noff[l];
                const float gl = net.gam[l];
                const float X = __fmaf_ru(gl, Nn, Ee);
                float hn[SM_MAXW];
                float ns = 0.f, us = 0.f;
                for (int i = 0; i < N; ++i) {
                    float acc = 0.f;
                    const float* w = &S.W[l][i * K];
                    for (int k = 0; k < K; ++k) acc = fmaf(h[k], w[k], acc);
                    const int gi = off + i;
                    const float ub = S.ub32[gi];
                    const float u = ub + acc;
                    const float bound = __fmaf_ru(S.rn[l][i], X, S.thr[gi]);
                    if (!(__fmul_rd(fabsf(u), 1.f - 0x1p-22f) > bound)) {
                        if (cov) unc = true;
                    } else if ((u >= 0.f) != (ub >= 0.f)) {
                        if (fcnt[l] < SM_FCAP) flist[l][fcnt[l]] = (short)i;
                        ++fcnt[l];
                        if (cov) atomicOr(&S.cflip[gi >> 5], 1u << (gi & 31));
                    }
                    if (l < L) {
                        const float dh = act_delta_s(net.act, acc, u, S.c1[gi], S.c2[gi]);
                        ns = fmaf(dh, dh, ns);
                        us = fmaf(u, u, us);
                        hn[i] = dh;
                    } else {
                        hn[i] = u;
                    }
                }
                for (int i = 0; i < N; ++i) h[i] = hn[i];
                if (l < L) {
                    const float Nl = norm_up_s(ns);
                    float El = __fmaf_ru(__fmul_ru(net.lamfrob[l], gl), Nn, Q.kvec[l]);
                    El = __fmaf_ru(net.lamsig[l], Ee, El);
                    El = __fmaf_ru(0x1p-24f, Nl, El);
                    if (net.act == ACT_SIGMOID) El = __fmaf_ru(0x1p-26f, norm_up_s(us), El);
                    Nn = Nl;
                    Ee = El;
                } else {
                    Nn = __fmul_ru(gl, Nn);  // gamma N_{L-1}: dot-product rounding
                }
            }
            // verdict (Eq. 10, or Eq. 11); h holds the layer-L values (or layer 1 when L = 1)
            const float gN = L > 1 ? Nn : 0.f, Ep = L > 1 ? Ee : 0.f;
            const float yD = h[D];
            const float rD = L > 1 ? S.rn[L][D] : 0.f;
            const float dD = S.dub[offL + D];
            bool unsafe = false, safe = true;
            if (Q.prop == PROP_THRESHOLD) {  // Eq. 11: per output ||W_o|| (gamma N + E) + dub_o
                const float V = (float)Q.V;
                bool da = false, db = false, oa = false, ob = true;
                for (int o = 0; o < HL; ++o) {
                    const float ro = L > 1 ? S.rn[L][o] : 0.f;
                    const float e = __fmaf_ru(ro, __fadd_ru(gN, Ep), __fadd_ru(S.dub[offL + o], (float)(2.0 * kTau)));
                    const int sd = thr_side(h[o], V, e);
                    if (o == D) { da = sd > 0; db = sd < 0; }
                    else { oa = oa || sd > 0; ob = ob && sd < 0; }
                }
                const int v = thr_verdict(da, db, oa, ob);
                unsafe = v == 1;
                safe = v == 0;
            } else {
                for (int o = 0; o < HL; ++o) {
                    if (o == D) continue;
                    const float yo = h[o];
                    const float diff = yD - yo;
                    const float ro = L > 1 ? S.rn[L][o] : 0.f;
                    const float pw = L > 1 ? net.pairw[D * HL + o] : 0.f;
                    float eb = __fmaf_ru(__fadd_ru(rD, ro), gN, __fadd_ru(__fadd_ru(dD, S.dub[offL + o]), (float)(2.0 * kTau)));
                    eb = __fmaf_ru(pw, Ep, eb);
                    eb = __fmaf_ru(0x1p-23f, __fadd_ru(__fadd_ru(fabsf(yD), fabsf(yo)), fabsf(diff)), eb);
                    if (diff < -eb) unsafe = true;
                    else if (!(diff > eb)) safe = false;
                }
            }
            vstate = unsafe ? 1 : (safe ? 0 : 2);
            if (Q.ss)
                for (int l = 1; l < L; ++l)
                    if (fcnt[l] == 1 && fcnt[l + 1] > SM_FCAP) ssover = true;
        }
        const bool bad = ok && (unc || vstate == 2 || ssover);
        queue_push_warp(out, bad, t, 0u, Q.cnt, out_level);
        const bool adv = ok && !bad && vstate == 1;
        if (!gather) {
            // the warp's points are 32 consecutive indices of one bitmap word
            const unsigned m = __ballot_sync(0xffffffffu, adv);
            if (m && lane == __ffs(m) - 1) {
                atomicAdd(&Q.cnt->n_adv, (unsigned long long)__popc(m));
                atomicMin(&Q.cnt->first, t);
                if (Q.bitmap && t < Q.bitmap_bits) atomicOr(&Q.bitmap[t >> 5], m);
            }
        } else if (adv) {
            record_adversarial(Q, t);
        }
        if (ok && !bad && Q.ss)
            for (int l = 1; l < L; ++l) {
                if (fcnt[l] != 1) continue;
                const int j = flist[l][0];
                const int Hn = net.dims[l + 1];
                for (int e = 0; e < fcnt[l + 1]; ++e)
                    set_bit_once(Q.ss, (unsigned long long)net.ssoff[l] + (unsigned long long)j * Hn + flist[l + 1][e]);
            }
        // time to verdict: a tile done, or this warp's queued points resolved
        if (gather) {
            const unsigned vm = __ballot_sync(0xffffffffu, ok);
            if (vm && lane == __ffs(vm) - 1) work_done(Q.cnt, __popc(vm));
        } else {
            __syncthreads();
            if (threadIdx.x == 0) work_done(Q.cnt, 1);
        }
    }
    __syncthreads();
    if (Q.flip && threadIdx.x < net.flip_words && threadIdx.x < SM_FW && S.cflip[threadIdx.x])
        atomicOr(&Q.flip[threadIdx.x], S.cflip[threadIdx.x]);
}

}  // namespace

bool small_supported(const NetView& net) {
    return net.L >= 1 && net.L <= SM_MAXL && net.hmax <= SM_MAXW && net.flip_words <= SM_FW;
}

int small_tile_points() { return SM_THREADS; }

void launch_small(const NetView& net, const QueryView* d_qs, const unsigned long long* tp,
                  unsigned long long n_tiles, const QEntry* gather, const unsigned long long* gc,
                  unsigned long long gcap, Queue out, int level, int n_sm, cudaStream_t st) {
    unsigned long long grid = (unsigned long long)n_sm * 4;
    if (!gather && n_tiles < grid) grid = n_tiles ? n_tiles : 1;
    k_small<<<(unsigned)grid, SM_THREADS, 0, st>>>(net, d_qs, tp, n_tiles, gather, gc, gcap, out, level);
}

}  // namespace vbmc
