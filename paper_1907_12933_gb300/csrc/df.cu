// df.cu -- double-float pass: points the FP32 bound could not decide, evaluated
// with FP32 pairs (hi + lo, about 48 significant bits) on the CUDA cores, which
// on this part run several times faster than FP64.
//
// Four points per CTA (each weight load serves all four). Layer 1 in FP64
// (incremental, Eq. 1). Layers 2..L on the
// deltas dh = h(point) - h(unperturbed), each weight (exact in FP32) times a
// pair (hi, lo): the product's rounding error is recovered exactly with an
// FMA, sums use TwoSum (Knuth), so a K-term dot product carries at most
// (K + 2) 2^-46 sum_j |w_j||dh_j| <= (K + 2) 2^-46 ||W_i|| ||dh|| of error.
// The error of the delta vector itself propagates with the spectral norm.
// A sign (Sec. III-B) or the class (Eq. 10, Eq. 11) is decided only when its value
// clears the bound by 2 tau; if anything is left undecided the whole point
// goes on to the FP64 pass and contributes nothing here.
#include "dev.cuh"
#include "launch.h"

#include <cfloat>

namespace vbmc {
namespace {

constexpr int TDF = 256;

__device__ __forceinline__ double act64(int act, double u) {
    if (act == ACT_SIGMOID) return 1.0 / (1.0 + exp(-u));
    if (act == ACT_RELU) return u > 0.0 ? u : 0.0;
    return u;
}

// M block-wide sums at once (one barrier pair for all of them); every thread
// gets the totals in v. red holds (blockDim.x / 32) x M doubles.
template <int M>
__device__ __forceinline__ void block_sums64(double (&v)[M], double* red) {
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < M; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int i = 0; i < M; ++i) red[w * M + i] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < M; ++i) {
        double t = 0.0;
        for (int k = 0; k < nw; ++k) t += red[k * M + i];
        v[i] = t;
    }
}

// PB points per CTA (one weight load serves all of them). Per point b: its
// potentials u[b], delta pair dh[b], certain sign changes fl[b].
template <int PB>
__global__ void __launch_bounds__(TDF)
k_df64(NetView net, const QueryView* __restrict__ qs, int nq, const QEntry* __restrict__ gather,
     const unsigned long long* __restrict__ gcount, unsigned long long gcap, Queue out,
     int out_level) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int total = net.total, hmax = net.hmax;
    double* u = reinterpret_cast<double*>(smem_raw);                       // [PB][total]
    float2* dh = reinterpret_cast<float2*>(u + (size_t)PB * total);        // [PB][hmax]
    unsigned char* fl = reinterpret_cast<unsigned char*>(dh + (size_t)PB * hmax);  // [PB][total]
    __shared__ double redm[(TDF / 32) * 2 * PB];
    __shared__ int nflip[PB][kMaxL + 2], only[PB][kMaxL + 2];
    __shared__ double dvs[PB][kMaxS];  // the point's input changes dv_p / 255 (FP64), once per pixel
    __shared__ int undecided[PB], valid[PB];
    __shared__ unsigned long long tpt[PB];
    __shared__ unsigned qpt[PB];

    unsigned long long n = *gcount;
    if (n > gcap) n = gcap;
    const int L = net.L;
    const double c46 = 0x1p-46, u52 = 0x1p-52;
    const double lam = net.act == ACT_SIGMOID ? 0.25 : 1.0;
    // compacted columns: one query whose set-up kept the non-"neg" neurons (their
    // change is 0 at every point of the box: dropped from the dense layers)
    const bool cmp = nq == 1 && qs[0].compact;
    for (unsigned long long e0 = (unsigned long long)blockIdx.x * PB; e0 < n;
         e0 += (unsigned long long)gridDim.x * PB) {
        if (threadIdx.x < PB) {
            const int b = threadIdx.x;
            const bool ok = e0 + b < n;
            valid[b] = ok;
            undecided[b] = 0;
            if (ok) {
                const QEntry en = gather[e0 + b];
                tpt[b] = en.t;
                qpt[b] = en.q;
                const QueryView& Q = qs[en.q];
                int d[kMaxS];
                decode_digits(en.t, Q.s, Q.R, d);
                for (int p = 0; p < Q.s; ++p) dvs[b][p] = (double)Q.dv[p * Q.R + d[p]] / 255.0;
            }
        }
        for (int e = threadIdx.x; e < PB * total; e += TDF) fl[e] = 0;  // neurons not computed: no change
        if (threadIdx.x < PB * (kMaxL + 2)) {
            nflip[threadIdx.x / (kMaxL + 2)][threadIdx.x % (kMaxL + 2)] = 0;
            only[threadIdx.x / (kMaxL + 2)][threadIdx.x % (kMaxL + 2)] = -1;
        }
        __syncthreads();
        double N[PB], E[PB];
        // ---- layer 1 in FP64; its signs are decided here
        const int H1 = net.dims[1];
        const int W1 = cmp ? qs[0].kc[1] : H1, cnt1 = cmp ? qs[0].kc[kMaxL + 2] : H1;
        double sq1[2 * PB];  // per point: ||dh_1||^2, ||err(dh_1)||^2 (this thread's terms)
        for (int b = 0; b < PB; ++b) {
            double nsq = 0.0, esq = 0.0;
            if (valid[b]) {
                const QueryView& Q = qs[qpt[b]];
                for (int jp = threadIdx.x; jp < W1; jp += TDF) {  // position jp holds neuron j
                    if (jp >= cnt1) {
                        dh[(size_t)b * hmax + jp] = make_float2(0.f, 0.f);
                        continue;
                    }
                    const int j = cmp ? Q.perm[jp] : jp;
                    const double ub = Q.ub[j];
                    double a = ub, mag = fabs(ub);
                    for (int p = 0; p < Q.s; ++p) {
                        // W_1[j][pix] from the transposed copy (compacted: the query's own rows
                        // by position): threads over j read contiguously
                        const float w = cmp ? Q.w1c[(size_t)p * H1 + jp] : net.WT[1][(size_t)Q.pix[p] * H1 + j];
                        const double term = (double)w * dvs[b][p];
                        a += term;
                        mag += fabs(term);
                    }
                    u[(size_t)b * total + j] = a;
                    // |a - exact| <= base error + rounding of the s additions and the terms
                    const double err = Q.eub[j] + (Q.s + 3) * u52 * mag;
                    const bool certain = fabs(a) > err + 2.0 * kTau && fabs(ub) >= kTau;
                    if (!certain && Q.flip) undecided[b] = 1;  // signs matter only for coverage
                    fl[(size_t)b * total + j] = certain && ((a >= 0.0) != (ub >= 0.0));
                    const double d = (L > 1 ? act64(net.act, a) : a) - Q.hb[j];
                    const float hi = (float)d;
                    dh[(size_t)b * hmax + jp] = make_float2(hi, (float)(d - (double)hi));
                    nsq += d * d;
                    const double ej = 2.0 * err + u52 * (fabs(a) + fabs(Q.hb[j])) * 4.0 + 0x1p-47 * fabs(d);
                    esq += ej * ej;
                }
            }
            sq1[2 * b] = nsq;
            sq1[2 * b + 1] = esq;
        }
        block_sums64<2 * PB>(sq1, redm);
#pragma unroll
        for (int b = 0; b < PB; ++b) {
            N[b] = sqrt(sq1[2 * b]) * (1.0 + 1e-12);
            E[b] = sqrt(sq1[2 * b + 1]) * (1.0 + 1e-12);
        }
        // ---- layers 2..L in double-float, PB points per weight load
        for (int l = 2; l <= L; ++l) {
            bool any = false;
            for (int b = 0; b < PB; ++b) any = any || (valid[b] && !undecided[b]);
            if (!any) break;
            const int NS = net.dims[l], off = net.noff[l];  // row stride of W_l^T
            const int K = cmp ? qs[0].kc[l - 1] : net.dims[l - 1];
            const int Nn = (cmp && l < L) ? qs[0].kc[l] : NS;
            const int cntN = (cmp && l < L) ? qs[0].kc[kMaxL + 1 + l] : NS;
            const float* WT = cmp ? qs[0].wtc[l] : net.WT[l];
            const double cK = (K + 2) * c46;
            double nsq2[PB], esq2[PB];
            for (int b = 0; b < PB; ++b) nsq2[b] = esq2[b] = 0.0;
            for (int i = threadIdx.x; i < Nn; i += TDF) {  // position i holds neuron io
                if (i >= cntN) continue;  // padding: change 0
                const int io = (cmp && l < L) ? qs[0].perm[off + i] : i;
                float S[PB], sl[PB];
#pragma unroll
                for (int b = 0; b < PB; ++b) S[b] = sl[b] = 0.f;
                // unrolled so that the weight loads of several j are in flight (each
                // point's sum still runs in order of j)
#pragma unroll 4
                for (int j = 0; j < K; ++j) {
                    const float w = WT[(size_t)j * NS + i];
#pragma unroll
                    for (int b = 0; b < PB; ++b) {
                        const float2 h = dh[(size_t)b * hmax + j];
                        const float pr = __fmul_rn(w, h.x);
                        float ep = __fmaf_rn(w, h.x, -pr);
                        ep = __fmaf_rn(w, h.y, ep);
                        const float tt = __fadd_rn(S[b], pr);
                        const float z = __fsub_rn(tt, S[b]);
                        const float er = __fadd_rn(__fsub_rn(S[b], __fsub_rn(tt, z)), __fsub_rn(pr, z));
                        S[b] = tt;
                        sl[b] = __fadd_rn(sl[b], __fadd_rn(er, ep));
                    }
                }
#pragma unroll
                for (int b = 0; b < PB; ++b) {
                    if (!valid[b] || undecided[b]) continue;
                    const QueryView& Q = qs[qpt[b]];
                    const double ub = Q.ub[off + io];
                    const double ui = ub + ((double)S[b] + (double)sl[b]);
                    u[(size_t)b * total + off + io] = ui;
                    const double err = (double)net.rownorm[l][io] * (cK * N[b] + E[b]) + Q.eub[off + io] +
                                       u52 * (fabs(ui) + fabs(ub));
                    const bool certain = fabs(ui) > err + 2.0 * kTau && fabs(ub) >= kTau;
                    if (!certain && Q.flip) undecided[b] = 1;  // signs matter only for coverage
                    fl[(size_t)b * total + off + io] = certain && ((ui >= 0.0) != (ub >= 0.0));
                    if (l < L) {
                        const double d = act64(net.act, ui) - Q.hb[off + io];
                        nsq2[b] += d * d;
                        const double ej = lam * (Q.eub[off + io] + u52 * (fabs(ui) + fabs(ub))) +
                                          Q.eub[off + io] + u52 * (fabs(ui) + fabs(Q.hb[off + io])) * 4.0 +
                                          0x1p-47 * fabs(d);
                        esq2[b] += ej * ej;
                    }
                }
            }
            __syncthreads();  // dh of layer l-1 fully consumed
            if (l < L) {
                double sq2[2 * PB];
                for (int b = 0; b < PB; ++b) {
                    if (valid[b]) {
                        const QueryView& Q = qs[qpt[b]];
                        for (int i = threadIdx.x; i < Nn; i += TDF) {
                            if (i >= cntN) {  // padding position
                                dh[(size_t)b * hmax + i] = make_float2(0.f, 0.f);
                                continue;
                            }
                            const int io = cmp ? Q.perm[off + i] : i;
                            const double d = act64(net.act, u[(size_t)b * total + off + io]) - Q.hb[off + io];
                            const float hi = (float)d;
                            dh[(size_t)b * hmax + i] = make_float2(hi, (float)(d - (double)hi));
                        }
                    }
                    sq2[2 * b] = nsq2[b];
                    sq2[2 * b + 1] = esq2[b];
                }
                block_sums64<2 * PB>(sq2, redm);
#pragma unroll
                for (int b = 0; b < PB; ++b) {
                    // ||err(dh_l)|| <= lambda (sigma_l E + (K+2) 2^-46 ||W_l||_F N) + per-element rounding
                    const double En = lam * ((double)net.sig[l] * E[b] + cK * (double)net.frob[l] * N[b]);
                    N[b] = sqrt(sq2[2 * b]) * (1.0 + 1e-12);
                    E[b] = (En + sqrt(sq2[2 * b + 1])) * (1.0 + 1e-12);
                }
            }
            __syncthreads();
        }
        // ---- verdict (Eq. 10 with the margin bound of each class pair, or Eq. 11): thread b
        if (threadIdx.x < PB && valid[threadIdx.x] && !undecided[threadIdx.x]) {
            const int b = threadIdx.x;
            const QueryView& Q = qs[qpt[b]];
            const int HL = net.dims[L], offL = net.noff[L];
            const double* y = u + (size_t)b * total + offL;
            const int D = Q.cnt->D;
            const double cK = (net.dims[L - 1] + 2) * c46;
            bool unsafe = false, safe = true;
            if (Q.prop == PROP_THRESHOLD) {  // Eq. 11: per output ||W_o|| (cK N + E) + eub_o
                const double V = Q.V;
                bool da = false, db = false, oa = false, ob = true;
                for (int o = 0; o < HL; ++o) {
                    const double e = (double)net.rownorm[L][o] * (cK * N[b] + (L > 1 ? E[b] : 0.0)) +
                                     Q.eub[offL + o] + 2.0 * kTau +
                                     u52 * 2.0 * (fabs(y[o]) + fabs(Q.ub[offL + o]) + fabs(V));
                    const int sd = y[o] - V > e ? 1 : (V - y[o] > e ? -1 : 0);
                    if (o == D) { da = sd > 0; db = sd < 0; }
                    else { oa = oa || sd > 0; ob = ob && sd < 0; }
                }
                const int vv = thr_verdict(da, db, oa, ob);
                unsafe = vv == 1;
                safe = vv == 0;
            }
            for (int o = 0; o < HL && Q.prop != PROP_THRESHOLD; ++o) {
                if (o == D) continue;
                const double diff = y[D] - y[o];
                double eb = ((double)net.rownorm[L][D] + (double)net.rownorm[L][o]) * cK * N[b] +
                            Q.eub[offL + D] + Q.eub[offL + o] + 2.0 * kTau +
                            u52 * 2.0 * (fabs(y[D]) + fabs(y[o]) + fabs(Q.ub[offL + D]) + fabs(Q.ub[offL + o]));
                eb += (L > 1 ? (double)net.pairw[D * HL + o] : 0.0) * E[b];
                if (diff < -eb) unsafe = true;
                else if (!(diff > eb)) safe = false;
            }
            if (!unsafe && !safe) undecided[b] = 1;
            if (!undecided[b] && unsafe) record_adversarial(Q, tpt[b]);
        }
        __syncthreads();
        for (int b = 0; b < PB; ++b) {
            if (!valid[b]) continue;
            const QueryView& Q = qs[qpt[b]];
            if (undecided[b]) {
                if (threadIdx.x == 0) queue_push(out, tpt[b], qpt[b], Q.cnt, out_level);
            } else {
                // sign changes and SS-Cover pairs; every decision here is certain (no ties)
                const unsigned char* flb = fl + (size_t)b * total;
                for (int nn = threadIdx.x; nn < total; nn += TDF) {
                    if (!flb[nn]) continue;
                    int l = 1;
                    while (l < L && nn >= net.noff[l + 1]) ++l;
                    atomicAdd(&nflip[b][l], 1);
                    atomicMax(&only[b][l], nn - net.noff[l]);
                    if (Q.flip) set_bit_once(Q.flip, nn);
                }
                __syncthreads();
                if (Q.ss) {
                    for (int l = 1; l < L; ++l) {
                        if (nflip[b][l] != 1) continue;
                        const int j = only[b][l], Hn = net.dims[l + 1], on = net.noff[l + 1];
                        for (int i = threadIdx.x; i < Hn; i += TDF)
                            if (flb[on + i])
                                set_bit_once(Q.ss, (unsigned long long)net.ssoff[l] + (unsigned long long)j * Hn + i);
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) work_done(Q.cnt, 1);  // time to verdict: this point is resolved
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ FP32 only
// The same pass for ReLU and identity nets with no FP64 arithmetic per point:
// potentials are FP32 pairs (hi + lo), every bound is FP32 rounded up. The
// FP64 base values (ub, hb, eub) are split into pairs once per neuron and
// shared by the CTA's PB points. Error of the pair operations (u = 2^-24):
//   two_sum(a, b): exact (Knuth);
//   df_add(a, b) = two_sum(two_sum(a_hi, b_hi) + (a_lo + b_lo)): at most
//     2.01 u (|a_lo| + |b_lo|) + u^2 (|a| + |b|), i.e. 2^-46 (|a| + |b|) for
//     normalised pairs (|lo| <= u |hi|);
//   the dot products (as above) with an unnormalised lo sum: (K + 2) 2^-45
//     sum_j |w_j||dh_j| covers both the sum and the pair addition after it.
// Potentials within the tie band 2 tau (tau = 1e-9) of 0 are left to the
// FP64 pass as before; these bounds are about 1e-12 relative, far inside it.

__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float2 s = two_sum(a.x, b.x);
    return two_sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}

// an FP64 value as a pair: |v - (hi + lo)| <= 2^-48 |v|
__device__ __forceinline__ float2 split64(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// M block-wide sums of non-negative terms, rounded up (upper bounds); every
// thread gets the totals. red holds (blockDim.x / 32) x M floats.
template <int M>
__device__ __forceinline__ void block_sums_ru(float (&v)[M], float* red) {
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < M; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] = __fadd_ru(v[i], __shfl_xor_sync(0xffffffffu, v[i], o));
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int i = 0; i < M; ++i) red[w * M + i] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < M; ++i) {
        float t = 0.f;
        for (int k = 0; k < nw; ++k) t = __fadd_ru(t, red[k * M + i]);
        v[i] = t;
    }
}

// Threads per position of a round of Nn positions with K inputs: a round of at
// most half a block (a narrow layer, or a layer's last round) splits its dot
// products into chunks of k.
__device__ __forceinline__ int df_split(int Nn, int K) {
    if (2 * Nn > TDF || K < 64) return 1;
    const int ks = TDF / Nn;
    return ks < 32 ? ks : 32;
}

__device__ __forceinline__ float abs_up(float2 a) { return __fmul_ru(fabsf(a.x), 1.f + 0x1p-22f); }

template <int PB>
__global__ void __launch_bounds__(TDF)
k_df32(NetView net, const QueryView* __restrict__ qs, int nq, const QEntry* __restrict__ gather,
       const unsigned long long* __restrict__ gcount, unsigned long long gcap, Queue out,
       int out_level) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int total = net.total, hmax = net.hmax;
    // u: potentials of every layer as pairs (hidden layers: after the layer's pass,
    // the delta dh = act(u) - hb in place of the potential); fl: certain changes
    float2* u = reinterpret_cast<float2*>(smem_raw);                        // [PB][total]
    float2* dh = u + (size_t)PB * total;                                    // [PB][hmax]
    unsigned char* fl = reinterpret_cast<unsigned char*>(dh + (size_t)PB * hmax);  // [PB][total]
    __shared__ float redm[(TDF / 32) * 2 * PB];
    __shared__ float2 part[PB][TDF];  // narrow layers: the chunk sums of each position
    __shared__ int nflip[PB][kMaxL + 2], only[PB][kMaxL + 2];
    __shared__ float2 dvs[PB][kMaxS];  // dv_p / 255 as a pair (|error| <= 2^-48 of it)
    __shared__ float dvm[PB][kMaxS];   // an upper bound of |dv_p / 255|
    __shared__ int undecided[PB], valid[PB];
    __shared__ unsigned long long tpt[PB];
    __shared__ unsigned qpt[PB];

    unsigned long long n = *gcount;
    if (n > gcap) n = gcap;
    const int L = net.L;
    const bool relu = net.act == ACT_RELU;
    const float tau2 = __double2float_ru(2.0 * kTau);  // >= 2 tau
    // compacted columns: one query whose set-up kept the non-"neg" neurons (their
    // change is 0 at every point of the box: dropped from the dense layers)
    const bool cmp = nq == 1 && qs[0].compact;
    for (unsigned long long e0 = (unsigned long long)blockIdx.x * PB; e0 < n;
         e0 += (unsigned long long)gridDim.x * PB) {
        if (threadIdx.x < PB) {
            const int b = threadIdx.x;
            const bool ok = e0 + b < n;
            valid[b] = ok;
            undecided[b] = 0;
            if (ok) {
                const QEntry en = gather[e0 + b];
                tpt[b] = en.t;
                qpt[b] = en.q;
                const QueryView& Q = qs[en.q];
                int d[kMaxS];
                decode_digits(en.t, Q.s, Q.R, d);
                for (int p = 0; p < Q.s; ++p) {
                    const double v = (double)Q.dv[p * Q.R + d[p]] / 255.0;
                    dvs[b][p] = split64(v);
                    dvm[b][p] = __double2float_ru(fabs(v));
                }
            }
        }
        for (int e = threadIdx.x; e < PB * total; e += TDF) fl[e] = 0;  // neurons not computed: no change
        if (threadIdx.x < PB * (kMaxL + 2)) {
            nflip[threadIdx.x / (kMaxL + 2)][threadIdx.x % (kMaxL + 2)] = 0;
            only[threadIdx.x / (kMaxL + 2)][threadIdx.x % (kMaxL + 2)] = -1;
        }
        __syncthreads();
        float N[PB], E[PB];
        // ---- layer 1 (Eq. 1 on the s changed pixels); its signs are decided here
        {
            const int H1 = net.dims[1];
            const int W1 = cmp ? qs[0].kc[1] : H1, cnt1 = cmp ? qs[0].kc[kMaxL + 2] : H1;
            float sq[2 * PB];  // per point: ||dh_1||^2, ||err(dh_1)||^2 (this thread's terms)
#pragma unroll
            for (int i = 0; i < 2 * PB; ++i) sq[i] = 0.f;
            for (int jp = threadIdx.x; jp < W1; jp += TDF) {  // position jp holds neuron j
                if (jp >= cnt1) {  // padding position: change 0
#pragma unroll
                    for (int b = 0; b < PB; ++b) dh[(size_t)b * hmax + jp] = make_float2(0.f, 0.f);
                    continue;
                }
                unsigned cq = ~0u;  // the query whose neuron constants are loaded
                int j = jp;
                float2 ubd = make_float2(0.f, 0.f), nhb = make_float2(0.f, 0.f);
                float eubu = 0.f;
                bool ubpos = false, ubbig = false;
#pragma unroll
                for (int b = 0; b < PB; ++b) {
                    if (!valid[b]) continue;
                    const QueryView& Q = qs[qpt[b]];
                    if (qpt[b] != cq) {
                        cq = qpt[b];
                        j = cmp ? Q.perm[jp] : jp;
                        const double ub = Q.ub[j];
                        ubd = split64(ub);
                        nhb = split64(-Q.hb[j]);
                        eubu = __double2float_ru(Q.eub[j]);
                        ubpos = ub >= 0.0;
                        ubbig = fabs(ub) >= kTau;
                    }
                    // du = sum_p W_1[j][pix_p] (dv_p / 255), the products' errors kept in sl
                    float S = 0.f, sl = 0.f, mag = 0.f;
                    for (int p = 0; p < Q.s; ++p) {
                        // W_1[j][pix] from the transposed copy (compacted: the query's own rows
                        // by position): threads over j read contiguously
                        const float w = cmp ? Q.w1c[(size_t)p * H1 + jp] : net.WT[1][(size_t)Q.pix[p] * H1 + j];
                        const float2 h = dvs[b][p];
                        const float pr = __fmul_rn(w, h.x);
                        float ep = __fmaf_rn(w, h.x, -pr);
                        ep = __fmaf_rn(w, h.y, ep);
                        const float2 t = two_sum(S, pr);
                        S = t.x;
                        sl = __fadd_rn(sl, __fadd_rn(t.y, ep));
                        mag = __fmaf_ru(fabsf(w), dvm[b][p], mag);
                    }
                    const float2 a = df_add(ubd, make_float2(S, sl));
                    // |a - exact| <= eub + (s + 3) 2^-45 mag (the sum; dv_p / 255 as pairs)
                    //                + 2^-44 (|ub| + |a|) (the pair addition; ub as a pair)
                    float err = __fmaf_ru((float)(Q.s + 3) * 0x1p-45f, mag, eubu);
                    err = __fmaf_ru(0x1p-44f, __fadd_ru(abs_up(ubd), abs_up(a)), err);
                    const bool certain = __fmul_rd(fabsf(a.x), 1.f - 0x1p-22f) > __fadd_ru(err, tau2) && ubbig;
                    if (!certain && Q.flip) undecided[b] = 1;  // signs matter only for coverage
                    fl[(size_t)b * total + j] = certain && ((a.x >= 0.f) != ubpos);
                    u[(size_t)b * total + j] = a;
                    // dh_1 = act(a) - hb (ReLU: a - hb where a > 0, else -hb)
                    const float2 d = (relu && !(a.x > 0.f)) ? nhb : df_add(a, nhb);
                    dh[(size_t)b * hmax + jp] = d;
                    sq[2 * b] = __fmaf_ru(d.x, d.x, sq[2 * b]);
                    // |d - exact| <= err (of a) + eub (of hb) + 2^-44 (|a| + |hb|) (the subtraction)
                    const float ej = __fmaf_ru(0x1p-44f, __fadd_ru(abs_up(a), abs_up(nhb)), __fmul_ru(2.f, err));
                    sq[2 * b + 1] = __fmaf_ru(ej, ej, sq[2 * b + 1]);
                }
            }
            block_sums_ru<2 * PB>(sq, redm);
#pragma unroll
            for (int b = 0; b < PB; ++b) {
                N[b] = __fmul_ru(__fsqrt_ru(sq[2 * b]), 1.f + 0x1p-20f);  // |d| <= |d_hi| (1 + 2^-24)
                E[b] = __fmul_ru(__fsqrt_ru(sq[2 * b + 1]), 1.f + 0x1p-20f);
            }
        }
        // ---- layers 2..L: pair dot products, PB points per weight load
        for (int l = 2; l <= L; ++l) {
            bool any = false;
            for (int b = 0; b < PB; ++b) any = any || (valid[b] && !undecided[b]);
            if (!any) break;
            const int NS = net.dims[l], off = net.noff[l];  // row stride of W_l^T
            const int K = cmp ? qs[0].kc[l - 1] : net.dims[l - 1];
            const int Nn = (cmp && l < L) ? qs[0].kc[l] : NS;
            const int cntN = (cmp && l < L) ? qs[0].kc[kMaxL + 1 + l] : NS;
            const float* WT = cmp ? qs[0].wtc[l] : net.WT[l];
            // positions run in rounds of TDF; a round of at most half a block (the
            // last one) splits each dot product over KS <= 32 threads
            const int remL = Nn % TDF;
            const bool anysplit = remL != 0 && df_split(remL, K) > 1;
            const float cK = (float)(K + 2 + (anysplit ? 32 : 0)) * 0x1p-45f;
            float X[PB];  // cK N + E: with ||W_i||, the propagated and summation error of u_i
#pragma unroll
            for (int b = 0; b < PB; ++b) X[b] = __fmaf_ru(cK, N[b], E[b]);
            float sq[2 * PB];
#pragma unroll
            for (int i = 0; i < 2 * PB; ++i) sq[i] = 0.f;
            // S + sl over k in [j0, j1) for position i, in order of k (loads of several k in flight)
            auto dot = [&](int i, int j0, int j1, float (&S)[PB], float (&sl)[PB]) {
#pragma unroll
                for (int b = 0; b < PB; ++b) S[b] = sl[b] = 0.f;
#pragma unroll 4
                for (int j = j0; j < j1; ++j) {
                    const float w = WT[(size_t)j * NS + i];
#pragma unroll
                    for (int b = 0; b < PB; ++b) {
                        const float2 h = dh[(size_t)b * hmax + j];
                        const float pr = __fmul_rn(w, h.x);
                        float ep = __fmaf_rn(w, h.x, -pr);
                        ep = __fmaf_rn(w, h.y, ep);
                        const float tt = __fadd_rn(S[b], pr);
                        const float z = __fsub_rn(tt, S[b]);
                        const float er = __fadd_rn(__fsub_rn(S[b], __fsub_rn(tt, z)), __fsub_rn(pr, z));
                        S[b] = tt;
                        sl[b] = __fadd_rn(sl[b], __fadd_rn(er, ep));
                    }
                }
            };
            // the sign tests and the next delta of position i (neuron io) from its sums
            auto finish = [&](int io, const float (&S)[PB], const float (&sl)[PB]) {
                const float rn = net.rownorm[l][io];
                unsigned cq = ~0u;
                float2 ubd = make_float2(0.f, 0.f), nhb = make_float2(0.f, 0.f);
                float eubu = 0.f;
                bool ubpos = false, ubbig = false;
#pragma unroll
                for (int b = 0; b < PB; ++b) {
                    if (!valid[b] || undecided[b]) continue;
                    const QueryView& Q = qs[qpt[b]];
                    if (qpt[b] != cq) {
                        cq = qpt[b];
                        const double ub = Q.ub[off + io];
                        ubd = split64(ub);
                        if (l < L) nhb = split64(-Q.hb[off + io]);
                        eubu = __double2float_ru(Q.eub[off + io]);
                        ubpos = ub >= 0.0;
                        ubbig = fabs(ub) >= kTau;
                    }
                    const float2 a = df_add(ubd, make_float2(S[b], sl[b]));
                    // |a - exact| <= ||W_i|| (cK N + E) + eub + 2^-44 (|ub| + |a|)
                    float err = __fmaf_ru(rn, X[b], eubu);
                    err = __fmaf_ru(0x1p-44f, __fadd_ru(abs_up(ubd), abs_up(a)), err);
                    const bool certain = __fmul_rd(fabsf(a.x), 1.f - 0x1p-22f) > __fadd_ru(err, tau2) && ubbig;
                    if (!certain && Q.flip) undecided[b] = 1;  // signs matter only for coverage
                    fl[(size_t)b * total + off + io] = certain && ((a.x >= 0.f) != ubpos);
                    if (l < L) {
                        const float2 d = (relu && !(a.x > 0.f)) ? nhb : df_add(a, nhb);
                        u[(size_t)b * total + off + io] = d;  // the delta, moved into dh below
                        sq[2 * b] = __fmaf_ru(d.x, d.x, sq[2 * b]);
                        // the local error of d: eub and the pair addition of a, eub of hb, the
                        // subtraction (the dot product's error propagates as a vector below)
                        const float ej = __fmaf_ru(0x1p-44f, __fadd_ru(__fadd_ru(abs_up(ubd), abs_up(nhb)),
                                                                      __fmul_ru(2.f, abs_up(a))),
                                                   __fmul_ru(2.f, eubu));
                        sq[2 * b + 1] = __fmaf_ru(ej, ej, sq[2 * b + 1]);
                    } else {
                        u[(size_t)b * total + off + io] = a;  // output potentials for the verdict
                    }
                }
            };
            for (int i0 = 0; i0 < Nn; i0 += TDF) {
                const int rem = min(TDF, Nn - i0);
                const int KS = df_split(rem, K);  // threads per position in this round
                if (KS == 1) {
                    const int i = i0 + threadIdx.x;  // position i holds neuron io
                    if (i < Nn && i < cntN) {        // padding positions: change 0
                        float S[PB], sl[PB];
                        dot(i, 0, K, S, sl);
                        finish((cmp && l < L) ? qs[0].perm[off + i] : i, S, sl);
                    }
                } else {
                    // KS threads per position, each a contiguous chunk of k; the chunks'
                    // pairs are then added in chunk order (within the bound's split term)
                    const int Kc = (K + KS - 1) / KS;
                    {
                        const int i = i0 + threadIdx.x / KS, c = threadIdx.x % KS;
                        if (i < Nn && i < cntN && threadIdx.x / KS < rem) {
                            float S[PB], sl[PB];
                            dot(i, min(K, c * Kc), min(K, (c + 1) * Kc), S, sl);
#pragma unroll
                            for (int b = 0; b < PB; ++b) part[b][threadIdx.x] = make_float2(S[b], sl[b]);
                        }
                    }
                    __syncthreads();
                    const int i = i0 + threadIdx.x;
                    if (threadIdx.x < rem && i < cntN) {
                        float S[PB], sl[PB];
#pragma unroll
                        for (int b = 0; b < PB; ++b) {
                            float2 acc = make_float2(0.f, 0.f);
                            for (int c = 0; c < KS; ++c) acc = df_add(acc, part[b][threadIdx.x * KS + c]);
                            S[b] = acc.x;
                            sl[b] = acc.y;
                        }
                        finish((cmp && l < L) ? qs[0].perm[off + i] : i, S, sl);
                    }
                }
            }
            __syncthreads();  // dh of layer l-1 fully consumed
            if (l < L) {
                for (int b = 0; b < PB; ++b) {
                    if (!valid[b]) continue;
                    for (int i = threadIdx.x; i < Nn; i += TDF) {
                        if (i >= cntN) {  // padding position
                            dh[(size_t)b * hmax + i] = make_float2(0.f, 0.f);
                            continue;
                        }
                        const int io = cmp ? qs[0].perm[off + i] : i;
                        dh[(size_t)b * hmax + i] = u[(size_t)b * total + off + io];
                    }
                }
                block_sums_ru<2 * PB>(sq, redm);
#pragma unroll
                for (int b = 0; b < PB; ++b) {
                    // ||err(dh_l)|| <= sigma_l E + cK ||W_l||_F N + ||local errors|| (ReLU, identity: 1-Lipschitz)
                    const float En = __fmaf_ru(net.sig[l], E[b], __fmul_ru(__fmul_ru(cK, net.frob[l]), N[b]));
                    N[b] = __fmul_ru(__fsqrt_ru(sq[2 * b]), 1.f + 0x1p-20f);
                    E[b] = __fmul_ru(__fadd_ru(En, __fsqrt_ru(sq[2 * b + 1])), 1.f + 0x1p-20f);
                }
            }
            __syncthreads();
        }
        // ---- verdict (Eq. 10 with the margin bound of each class pair, or Eq. 11): thread b
        if (threadIdx.x < PB && valid[threadIdx.x] && !undecided[threadIdx.x]) {
            const int b = threadIdx.x;
            const QueryView& Q = qs[qpt[b]];
            const int HL = net.dims[L], offL = net.noff[L];
            const float2* y = u + (size_t)b * total + offL;
            const int D = Q.cnt->D;
            // the output layer's summation term (a split layer adds at most 32 to K + 2)
            const float cKL = (float)(net.dims[L - 1] + 2 + 32) * 0x1p-45f;
            const float cN = __fmul_ru(cKL, N[b]);
            bool unsafe = false, safe = true;
            if (Q.prop == PROP_THRESHOLD) {  // Eq. 11: per output ||W_o|| (cK N + E) + eub_o
                const double V = Q.V;
                const float2 nV = split64(-V);
                const float aV = __double2float_ru(fabs(V));
                bool da = false, db = false, oa = false, ob = true;
                for (int o = 0; o < HL; ++o) {
                    float e = __fmaf_ru(net.rownorm[L][o], __fadd_ru(cN, E[b]),
                                        __fadd_ru(__double2float_ru(Q.eub[offL + o]), tau2));
                    e = __fmaf_ru(0x1p-43f, __fadd_ru(__fadd_ru(abs_up(y[o]), aV),
                                                      __double2float_ru(fabs(Q.ub[offL + o]))), e);
                    const float2 df = df_add(y[o], nV);  // y_o - V
                    const bool clear = __fmul_rd(fabsf(df.x), 1.f - 0x1p-22f) > e;
                    const int sd = clear ? (df.x > 0.f ? 1 : -1) : 0;
                    if (o == D) { da = sd > 0; db = sd < 0; }
                    else { oa = oa || sd > 0; ob = ob && sd < 0; }
                }
                const int vv = thr_verdict(da, db, oa, ob);
                unsafe = vv == 1;
                safe = vv == 0;
            }
            for (int o = 0; o < HL && Q.prop != PROP_THRESHOLD; ++o) {
                if (o == D) continue;
                const float2 df = df_add(y[D], make_float2(-y[o].x, -y[o].y));  // y_D - y_o
                float eb = __fmaf_ru(__fadd_ru(net.rownorm[L][D], net.rownorm[L][o]), cN,
                                     __fadd_ru(__fadd_ru(__double2float_ru(Q.eub[offL + D]),
                                                         __double2float_ru(Q.eub[offL + o])), tau2));
                eb = __fmaf_ru(0x1p-43f,
                               __fadd_ru(__fadd_ru(abs_up(y[D]), abs_up(y[o])),
                                         __double2float_ru(fabs(Q.ub[offL + D]) + fabs(Q.ub[offL + o]))),
                               eb);
                eb = __fmaf_ru(net.pairw[D * HL + o], E[b], eb);
                const bool clear = __fmul_rd(fabsf(df.x), 1.f - 0x1p-22f) > eb;
                if (clear && df.x < 0.f) unsafe = true;
                else if (!(clear && df.x > 0.f)) safe = false;
            }
            if (!unsafe && !safe) undecided[b] = 1;
            if (!undecided[b] && unsafe) record_adversarial(Q, tpt[b]);
        }
        __syncthreads();
        for (int b = 0; b < PB; ++b) {
            if (!valid[b]) continue;
            const QueryView& Q = qs[qpt[b]];
            if (undecided[b]) {
                if (threadIdx.x == 0) queue_push(out, tpt[b], qpt[b], Q.cnt, out_level);
            } else {
                // sign changes and SS-Cover pairs; every decision here is certain (no ties)
                const unsigned char* flb = fl + (size_t)b * total;
                for (int nn = threadIdx.x; nn < total; nn += TDF) {
                    if (!flb[nn]) continue;
                    int l = 1;
                    while (l < L && nn >= net.noff[l + 1]) ++l;
                    atomicAdd(&nflip[b][l], 1);
                    atomicMax(&only[b][l], nn - net.noff[l]);
                    if (Q.flip) set_bit_once(Q.flip, nn);
                }
                __syncthreads();
                if (Q.ss) {
                    for (int l = 1; l < L; ++l) {
                        if (nflip[b][l] != 1) continue;
                        const int j = only[b][l], Hn = net.dims[l + 1], on = net.noff[l + 1];
                        for (int i = threadIdx.x; i < Hn; i += TDF)
                            if (flb[on + i])
                                set_bit_once(Q.ss, (unsigned long long)net.ssoff[l] + (unsigned long long)j * Hn + i);
                    }
                }
            }
            __syncthreads();
        }
        // time to verdict: the iteration's points are resolved (the queued ones stay
        // counted through their push), one count per query; a thread that decodes no
        // point reads them before the barrier and adds them after it, while the next
        // iteration decodes
        constexpr int kCntT = TDF - 1;
        static_assert(kCntT >= PB, "the counting thread decodes no point");
        unsigned cq[PB];
        unsigned long long cn[PB];
        int ncq = 0;
        if (threadIdx.x == kCntT) {
#pragma unroll
            for (int b = 0; b < PB; ++b) {
                if (!valid[b]) continue;
                int k = 0;
                while (k < ncq && cq[k] != qpt[b]) ++k;
                if (k == ncq) {
                    cq[ncq] = qpt[b];
                    cn[ncq++] = 0;
                }
                ++cn[k];
            }
        }
        __syncthreads();
        if (threadIdx.x == kCntT)
            for (int k = 0; k < ncq; ++k) work_done(qs[cq[k]].cnt, cn[k]);
    }
}

}  // namespace

void launch_df(const NetView& net, const QueryView* d_qs, int nq, const QEntry* gather,
               const unsigned long long* gather_count, unsigned long long gather_cap, Queue out,
               int out_level, int n_sm, cudaStream_t st) {
    constexpr int PB = 4;
    const size_t smem = PB * (sizeof(double) * net.total + sizeof(float2) * net.hmax + (size_t)net.total);
    const int per_sm = (net.df_ctas >= 1 && net.df_ctas <= 32) ? net.df_ctas : 4;
    const unsigned grid = (unsigned)(n_sm * per_sm);
    if (net.act == ACT_SIGMOID || net.L < 2) {  // FP64 where a pair activation or bound is not built
        cudaFuncSetAttribute(k_df64<PB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_df64<PB><<<grid, TDF, smem, st>>>(net, d_qs, nq, gather, gather_count, gather_cap, out, out_level);
    } else {
        cudaFuncSetAttribute(k_df32<PB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_df32<PB><<<grid, TDF, smem, st>>>(net, d_qs, nq, gather, gather_count, gather_cap, out, out_level);
    }
}

}  // namespace vbmc
