// prologue.cu -- per-query set-up that every pass over the points uses.
//
//  * k_pro_init:   validate the pixel list, build the clipped step table
//                  dv[p][d] = clamp(v_p + d - k, 0, 255) - v_p, reset counters
//  * k_pro_layer:  FP64 activation potentials of the unperturbed image, one
//                  layer per launch (Eq. 1; Eq. 2 or ReLU on hidden layers)
//  * k_pro_tables: layer-1 delta tables tab[p][d][j] = W_1[j][p] * dv[p][d] / 255,
//                  so a point's layer-1 potential is ub_1 + sum_p tab[p][d_p]
//                  (the incremental first layer: s table adds instead of an
//                  H_0-long dot product per neuron)
//  * k_pro_finish: class D and margin of the unperturbed image, and the
//                  per-neuron constants of the screens' error bounds
#include "dev.cuh"
#include "launch.h"

#include <cfloat>

namespace vbmc {

__global__ void k_pro_init(NetView net, QueryView* qs, int nq) {
    QueryView& Q = qs[blockIdx.x];
    const int H0 = net.dims[0];
    if (threadIdx.x == 0) {
        bool ok = Q.s >= 0 && Q.s <= kMaxS;
        for (int p = 0; p < Q.s && ok; ++p) {
            int v = Q.pix_in[p];
            ok = v >= 0 && v < H0;
            for (int r = 0; r < p && ok; ++r) ok = Q.pix_in[r] != v;
        }
        Counters* c = Q.cnt;
        c->n_adv = 0;
        c->first = ~0ull;
        c->n_ties = 0;
        c->n_q[0] = c->n_q[1] = c->n_q[2] = c->n_q[3] = 0;
        c->n_points = Q.filter ? 0ull : Q.hi - Q.lo;  // with a filter the passes count
        c->err = ok ? 0u : DERR_PIXELS;
        c->D = 0;
        c->base_margin = 0.0;
        c->t0 = globaltimer_ns();
        c->t_final = 0;
        c->work = Q.ntiles;
        for (int p = 0; p < Q.s; ++p) {
            int v = Q.pix_in[p];
            Q.pix[p] = (ok && v >= 0 && v < H0) ? v : 0;  // never index out of range
        }
    }
    // results start from zero on every call
    if (Q.flip)
        for (int w = threadIdx.x; w < net.flip_words; w += blockDim.x) Q.flip[w] = Q.flip_tie[w] = 0u;
    if (Q.ss)
        for (int w = threadIdx.x; w < net.ss_words; w += blockDim.x) Q.ss[w] = Q.ss_tie[w] = 0u;
    if (Q.bitmap && Q.hi > 0) {
        const unsigned long long nw = (Q.hi + 31) / 32;
        uint4* b4 = reinterpret_cast<uint4*>(Q.bitmap);
        for (unsigned long long w = threadIdx.x; w < nw / 4; w += blockDim.x) b4[w] = make_uint4(0, 0, 0, 0);
        for (unsigned long long w = (nw / 4) * 4 + threadIdx.x; w < nw; w += blockDim.x) Q.bitmap[w] = 0u;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < Q.s * Q.R; e += blockDim.x) {
        int p = e / Q.R, d = e % Q.R;
        int v = Q.image[Q.pix[p]];
        int w = v + d - Q.k;
        w = w < 0 ? 0 : (w > 255 ? 255 : w);
        Q.dv[e] = w - v;
    }
}

__device__ __forceinline__ double act64(int act, double u) {
    if (act == ACT_SIGMOID) return 1.0 / (1.0 + exp(-u));  // Eq. 2
    if (act == ACT_RELU) return u > 0.0 ? u : 0.0;
    return u;
}

// One warp per neuron i of layer l; lanes stride over the inputs. Also bounds
// the FP64 error of the result: rounding of the K products and sums,
// (K + 2) 2^-53 (sum_j |w_j h_j| + |b|), plus the input errors propagated,
// sum_j |w_j| e_j (the activations are 1-Lipschitz).
__global__ void k_pro_layer(NetView net, QueryView* qs, int nq, int l) {
    const QueryView& Q = qs[blockIdx.y];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + warp;
    const int K = net.dims[l - 1], N = net.dims[l];
    if (i >= N) return;
    const float* Wr = net.W[l] + (size_t)i * K;
    double acc = 0.0, mag = 0.0, prop = 0.0;
    if (l == 1) {
        for (int j = lane; j < K; j += 32) {
            const double p = (double)Wr[j] * ((double)Q.image[j] / 255.0);
            acc += p;
            mag += fabs(p);
        }
    } else {
        const double* h = Q.hb + net.noff[l - 1];
        const double* eh = Q.eub + net.noff[l - 1];
        for (int j = lane; j < K; j += 32) {
            const double p = (double)Wr[j] * h[j];
            acc += p;
            mag += fabs(p);
            prop += fabs((double)Wr[j]) * eh[j];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        mag += __shfl_xor_sync(0xffffffffu, mag, o);
        prop += __shfl_xor_sync(0xffffffffu, prop, o);
    }
    if (lane == 0) {
        const double bi = (double)net.b[l][i];
        double u = acc + bi;
        Q.ub[net.noff[l] + i] = u;
        Q.hb[net.noff[l] + i] = (l < net.L) ? act64(net.act, u) : u;
        // (x/255 carries one more rounding on layer 1; activations add 2^-50 |u|)
        const double e = ((K + 4) * 0x1p-53 * (mag + fabs(bi)) + prop + 0x1p-50 * fabs(u)) * (1.0 + 1e-9);
        Q.eub[net.noff[l] + i] = e;
    }
}

__global__ void k_pro_tables(NetView net, QueryView* qs, int nq) {
    const QueryView& Q = qs[blockIdx.y];
    const int e = blockIdx.x;  // e = p * R + d
    if (e >= Q.s * Q.R) return;
    const int p = e / Q.R;
    const int H0 = net.dims[0], H1 = net.dims[1];
    const double step = (double)Q.dv[e] / 255.0;
    const float* W1 = net.W[1];
    const int col = Q.pix[p];
    for (int j = threadIdx.x; j < H1; j += blockDim.x)
        Q.tab[(size_t)e * H1 + j] = (float)((double)W1[(size_t)j * H0 + col] * step);
}

// Rounded-up float of a non-negative double.
__device__ __forceinline__ float up(double x) { return __double2float_ru(x); }

__device__ __forceinline__ double block_sum(double v, double* red) {
    // blockDim.x is a multiple of 32 and at most 1024
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// Screen constants. With fl() the fp32 rounding and u = 2^-24:
//  dub_n   = |fl(ub_n) - ub_n| + eub_n   (+ e1_j on layer 1); eub bounds the FP64
//            error of ub itself, so every screen decision holds in exact arithmetic
//  thr_n   = dub_n + 2 tau, infinite when |ub_n| < tau (every evaluation of n is
//            a sign tie)
//  e1_j    = (gamma_{s+2} + 2u) * sum_p max_d |tab[p][d][j]|, the layer-1 table-sum error
//  ReLU:     c1 = 0, c2 = -fl(ub) when ub >= 0; c1 = fl(ub), c2 = 0 otherwise, so the
//            output change is max(du + c1, c2)
//  sigmoid / identity: c1 = fl(ub), c2 = fl(hb)
//  kvec[l] = norm of the point-independent part of the layer-l output error
__global__ void k_pro_finish(NetView net, QueryView* qs, int nq) {
    __shared__ double red[33];
    QueryView& Q = qs[blockIdx.x];
    const int L = net.L, HL = net.dims[L];
    const double* y = Q.ub + net.noff[L];
    if (threadIdx.x == 0) {
        int D = 0;
        for (int i = 1; i < HL; ++i)
            if (y[i] > y[D]) D = i;
        double mx = -DBL_MAX;
        for (int i = 0; i < HL; ++i)
            if (i != D && y[i] > mx) mx = y[i];
        Q.cnt->D = D;
        // Eq. 10 margin, or max(y_D - V, V - max_{i!=D} y_i) for Eq. 11
        Q.cnt->base_margin = Q.prop == PROP_THRESHOLD ? fmax(y[D] - Q.V, Q.V - mx) : y[D] - mx;
    }
    const double u24 = 0x1p-24;
    const int s = Q.s;
    const double gam = (s + 2) * u24 / (1.0 - (s + 2) * u24) + 2.0 * u24;
    for (int l = 1; l <= L; ++l) {
        const int H = net.dims[l];
        double ss_a = 0.0, ss_b = 0.0;  // squared norms of per-neuron constant errors
        for (int i = threadIdx.x; i < H; i += blockDim.x) {
            const int n = net.noff[l] + i;
            const double ub = Q.ub[n], hb = Q.hb[n];
            const float ub32 = __double2float_rn(ub);
            const double dub = fabs((double)ub32 - ub) + Q.eub[n];
            double e1 = 0.0;
            if (l == 1) {
                double b1 = 0.0;
                for (int p = 0; p < s; ++p) {
                    double mx = 0.0;
                    for (int d = 0; d < Q.R; ++d)
                        mx = fmax(mx, fabs((double)Q.tab[((size_t)p * Q.R + d) * H + i]));
                    b1 += mx;
                }
                e1 = gam * b1 * (1.0 + 1e-12);
            }
            const bool base_tie = fabs(ub) < kTau;
            Q.ub32[n] = ub32;
            Q.dub[n] = up(dub + e1);
            Q.thr[n] = base_tie ? INFINITY : up(dub + e1 + 2.0 * kTau);
            if (net.act == ACT_RELU) {
                Q.c1[n] = ub >= 0.0 ? 0.0f : ub32;
                Q.c2[n] = ub >= 0.0 ? -ub32 : 0.0f;
            } else {
                Q.c1[n] = ub32;
                Q.c2[n] = __double2float_rn(hb);
            }
            const double dhb = fabs((double)__double2float_rn(hb) - hb) + Q.eub[n];
            if (l < L) {
                if (net.act == ACT_RELU) {
                    ss_a += (e1 + dub) * (e1 + dub);
                } else if (net.act == ACT_SIGMOID) {
                    ss_a += (e1 + dub) * (e1 + dub);
                    ss_b += dhb * dhb;
                } else {
                    ss_a += e1 * e1;
                }
            }
        }
        double na = sqrt(block_sum(ss_a, red));
        double nb = sqrt(block_sum(ss_b, red));
        if (threadIdx.x == 0) {
            double kv = 0.0;
            if (l < L) {
                if (net.act == ACT_RELU) kv = na;
                else if (net.act == ACT_SIGMOID) kv = 0.25 * na + nb + sqrt((double)H) * 8.0 * u24;
                else kv = na;
            }
            Q.kvec[l] = up(kv * (1.0 + 1e-9));
        }
        __syncthreads();
    }
}

// Time to verdict of queries whose work count never reached zero inside a pass
// (no screen tiles: empty ranges and the FP64-only path): the end of the last pass.
__global__ void k_stamp_final(QueryView* qs, int nq) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    Counters* c = qs[q].cnt;
    if (c->t_final == 0) c->t_final = globaltimer_ns();
}

void launch_stamp_final(QueryView* d_qs, int nq, cudaStream_t st) {
    k_stamp_final<<<(nq + 127) / 128, 128, 0, st>>>(d_qs, nq);
}

void launch_pro_init(const NetView& net, QueryView* d_qs, int nq, cudaStream_t st) {
    k_pro_init<<<nq, 256, 0, st>>>(net, d_qs, nq);
}

void launch_pro_layer(const NetView& net, QueryView* d_qs, int nq, int l, cudaStream_t st) {
    k_pro_layer<<<dim3((net.dims[l] + 7) / 8, nq), 256, 0, st>>>(net, d_qs, nq, l);
}

void launch_prologue(const NetView& net, QueryView* d_qs, int nq, int max_sr, cudaStream_t st) {
    k_pro_init<<<nq, 256, 0, st>>>(net, d_qs, nq);
    for (int l = 1; l <= net.L; ++l) {
        dim3 grid((net.dims[l] + 7) / 8, nq);
        k_pro_layer<<<grid, 256, 0, st>>>(net, d_qs, nq, l);
    }
    if (max_sr > 0) k_pro_tables<<<dim3(max_sr, nq), 256, 0, st>>>(net, d_qs, nq);
    k_pro_finish<<<nq, 256, 0, st>>>(net, d_qs, nq);
}

}  // namespace vbmc
