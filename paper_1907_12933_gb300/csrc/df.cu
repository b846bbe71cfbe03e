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
k_df(NetView net, const QueryView* __restrict__ qs, int nq, const QEntry* __restrict__ gather,
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

}  // namespace

void launch_df(const NetView& net, const QueryView* d_qs, int nq, const QEntry* gather,
               const unsigned long long* gather_count, unsigned long long gather_cap, Queue out,
               int out_level, int n_sm, cudaStream_t st) {
    constexpr int PB = 4;
    const size_t smem = PB * (sizeof(double) * net.total + sizeof(float2) * net.hmax + (size_t)net.total);
    cudaFuncSetAttribute(k_df<PB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int per_sm = (net.df_ctas >= 1 && net.df_ctas <= 32) ? net.df_ctas : 4;
    k_df<PB><<<(unsigned)(n_sm * per_sm), TDF, smem, st>>>(net, d_qs, nq, gather, gather_count, gather_cap,
                                                          out, out_level);
}

}  // namespace vbmc
