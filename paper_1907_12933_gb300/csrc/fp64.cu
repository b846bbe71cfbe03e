// fp64.cu -- the final pass: points evaluated in FP64 on CUDA cores.
//
// One CTA per point. Layer 1 is incremental (ub_1 + sum_p W_1[:, p] dv_p / 255,
// Eq. 1), layers 2..L are full FP64 dot products over W_l^T (coalesced), the
// hidden outputs use sigmoid (Eq. 2) or ReLU. The point's results follow the
// definitions directly:
//   * margin m = y_D - max_{i != D} y_i; |m| < tau: tie (listed, not counted);
//     otherwise adversarial iff argmax(y) (lowest index) != D      (Eq. 10)
//   * sign(u) = [u >= 0]; neuron n is a sign tie at this point when |u_n| < tau
//     or |ub_n| < tau; a non-tie sign change sets its flip bit, a sign tie
//     sets its flip-tie bit                                         (Sec. III-B)
//   * SS-Cover of (j in layer l, i in layer l+1): certain when layer l has no
//     tie and exactly one change (j) and i changes without tie; pairs that
//     hold only under some resolution of the ties go to the SS-tie mask.
#include "dev.cuh"
#include "launch.h"

#include <cfloat>

namespace vbmc {
namespace {

constexpr int T64 = 256;

__device__ __forceinline__ double act64(int act, double u) {
    if (act == ACT_SIGMOID) return 1.0 / (1.0 + exp(-u));
    if (act == ACT_RELU) return u > 0.0 ? u : 0.0;
    return u;
}

__global__ void __launch_bounds__(T64)
k_fp64(NetView net, const QueryView* __restrict__ qs, const QEntry* __restrict__ gather,
       const unsigned long long* __restrict__ gather_count, unsigned long long gather_cap,
       unsigned long long range_lo, unsigned long long range_hi) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int total = net.total, hmax = net.hmax;
    double* u = reinterpret_cast<double*>(smem_raw);       // [total]
    double* h = u + total;                                   // [hmax]
    unsigned char* fl = reinterpret_cast<unsigned char*>(h + hmax);  // [total]
    unsigned char* ti = fl + total;                                   // [total]
    __shared__ int nflip[kMaxL + 2], ntie[kMaxL + 2], only[kMaxL + 2];
    __shared__ int dstep[kMaxS];
    __shared__ int skip;

    unsigned long long n;
    if (gather) {
        n = *gather_count;
        if (n > gather_cap) n = gather_cap;
    } else {
        n = range_hi - range_lo;
    }
    const int L = net.L;
    for (unsigned long long e = blockIdx.x; e < n; e += gridDim.x) {
        unsigned long long t;
        int qi;
        if (gather) {
            QEntry en = gather[e];
            t = en.t;
            qi = (int)en.q;
        } else {
            t = range_lo + e;
            qi = 0;
        }
        const QueryView& Q = qs[qi];
        if (threadIdx.x == 0) {
            int d[kMaxS];
            decode_digits(t, Q.s, Q.R, d);
            for (int p = 0; p < Q.s; ++p) dstep[p] = Q.dv[p * Q.R + d[p]];
            skip = !gather && Q.filter && !in_filter(Q, d);  // outside the L2 ball / shell
            if (!gather && Q.filter && !skip) atomicAdd(&Q.cnt->n_points, 1ull);
        }
        __syncthreads();
        if (skip) continue;
        if (threadIdx.x <= kMaxL + 1) {
            nflip[threadIdx.x] = 0;
            ntie[threadIdx.x] = 0;
            only[threadIdx.x] = -1;
        }
        __syncthreads();
        // layer 1, incremental in FP64
        {
            const int H0 = net.dims[0], H1 = net.dims[1];
            const float* W1 = net.W[1];
            for (int j = threadIdx.x; j < H1; j += T64) {
                double a = Q.ub[j];
                for (int p = 0; p < Q.s; ++p)
                    a += (double)W1[(size_t)j * H0 + Q.pix[p]] * ((double)dstep[p] / 255.0);
                u[j] = a;
                h[j] = (L > 1) ? act64(net.act, a) : a;
            }
        }
        __syncthreads();
        for (int l = 2; l <= L; ++l) {
            const int K = net.dims[l - 1], N = net.dims[l];
            const float* WT = net.WT[l];
            const float* b = net.b[l];
            const int off = net.noff[l];
            for (int i = threadIdx.x; i < N; i += T64) {
                double a = 0.0;
                for (int j = 0; j < K; ++j) a += (double)WT[(size_t)j * N + i] * h[j];
                u[off + i] = a + (double)b[i];
            }
            __syncthreads();
            if (l < L)
                for (int i = threadIdx.x; i < N; i += T64) h[i] = act64(net.act, u[off + i]);
            __syncthreads();
        }
        // signs, ties, changes
        for (int nn = threadIdx.x; nn < total; nn += T64) {
            const double ub = Q.ub[nn], ut = u[nn];
            const bool tie = fabs(ut) < kTau || fabs(ub) < kTau;
            const bool ch = ((ut >= 0.0) != (ub >= 0.0)) && !tie;
            fl[nn] = ch;
            ti[nn] = tie;
            int l = 1;
            while (l < L && nn >= net.noff[l + 1]) ++l;
            if (ch) {
                atomicAdd(&nflip[l], 1);
                atomicMax(&only[l], nn - net.noff[l]);
                if (Q.flip) set_bit_once(Q.flip, nn);
            }
            if (tie) {
                atomicAdd(&ntie[l], 1);
                if (Q.flip_tie) set_bit_once(Q.flip_tie, nn);
            }
        }
        __syncthreads();
        // SS-Cover pairs (j in l, i in l+1)
        if (Q.ss) {
            for (int l = 1; l < L; ++l) {
                const int Hl = net.dims[l], Hn = net.dims[l + 1];
                const int ol = net.noff[l], on = net.noff[l + 1];
                const bool certain = ntie[l] == 0 && nflip[l] == 1;
                if (!certain && ntie[l] == 0) continue;  // no flip or >= 2 certain flips
                if (!certain && nflip[l] >= 2) continue;
                for (int j = 0; j < Hl; ++j) {
                    bool cand;
                    if (certain || nflip[l] == 1) cand = (j == only[l]);
                    else cand = ti[ol + j];  // no certain flip, some ties: each tie may be the one
                    if (!cand) continue;
                    for (int i = threadIdx.x; i < Hn; i += T64) {
                        const unsigned long long bit = (unsigned long long)net.ssoff[l] +
                                                       (unsigned long long)j * Hn + i;
                        if (certain && fl[on + i]) set_bit_once(Q.ss, bit);
                        else if (fl[on + i] || ti[on + i]) set_bit_once(Q.ss_tie, bit);
                    }
                }
            }
        }
        // verdict
        if (threadIdx.x == 0) {
            const int HL = net.dims[L];
            const double* y = u + net.noff[L];
            const int D = Q.cnt->D;
            int am = 0;
            double mx = -DBL_MAX;
            for (int i = 0; i < HL; ++i) {
                if (y[i] > y[am]) am = i;
                if (i != D && y[i] > mx) mx = y[i];
            }
            // Eq. 10: m = y_D - max_{i!=D} y_i; Eq. 11: m = max(y_D - V, V - max_{i!=D} y_i),
            // negative iff y_D < V < some other output
            const bool thr = Q.prop == PROP_THRESHOLD;
            const double m = thr ? fmax(y[D] - Q.V, Q.V - mx) : y[D] - mx;
            if (thr) am = m < 0.0 ? -1 : D;
            if (fabs(m) < kTau) {
                unsigned long long k = atomicAdd(&Q.cnt->n_ties, 1ull);
                if (k < Q.ties_cap) Q.ties[k] = t;
                else atomicOr(&Q.cnt->err, DERR_TIES);
            } else if (am != D) {
                record_adversarial(Q, t);
            }
            if (gather) work_done(Q.cnt, 1);  // time to verdict: this queued point is resolved
        }
        __syncthreads();
    }
}

// FP64 margin of one point (for witnesses): y_D - max_{i != D} y_i.
__global__ void __launch_bounds__(T64)
k_margin64(NetView net, const QueryView* __restrict__ qs, unsigned long long t, double* out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* u = reinterpret_cast<double*>(smem_raw);
    double* h = u + net.total;
    __shared__ int dstep[kMaxS];
    const QueryView& Q = qs[0];
    const int L = net.L;
    if (threadIdx.x == 0) {
        int d[kMaxS];
        decode_digits(t, Q.s, Q.R, d);
        for (int p = 0; p < Q.s; ++p) dstep[p] = Q.dv[p * Q.R + d[p]];
    }
    __syncthreads();
    const int H0 = net.dims[0], H1 = net.dims[1];
    for (int j = threadIdx.x; j < H1; j += T64) {
        double a = Q.ub[j];
        for (int p = 0; p < Q.s; ++p)
            a += (double)net.W[1][(size_t)j * H0 + Q.pix[p]] * ((double)dstep[p] / 255.0);
        u[j] = a;
        h[j] = (L > 1) ? act64(net.act, a) : a;
    }
    __syncthreads();
    for (int l = 2; l <= L; ++l) {
        const int K = net.dims[l - 1], N = net.dims[l];
        for (int i = threadIdx.x; i < N; i += T64) {
            double a = 0.0;
            for (int j = 0; j < K; ++j) a += (double)net.WT[l][(size_t)j * N + i] * h[j];
            u[net.noff[l] + i] = a + (double)net.b[l][i];
        }
        __syncthreads();
        if (l < L)
            for (int i = threadIdx.x; i < N; i += T64) h[i] = act64(net.act, u[net.noff[l] + i]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double* y = u + net.noff[L];
        const int D = Q.cnt->D;
        double mx = -DBL_MAX;
        for (int i = 0; i < net.dims[L]; ++i)
            if (i != D && y[i] > mx) mx = y[i];
        *out = Q.prop == PROP_THRESHOLD ? fmax(y[D] - Q.V, Q.V - mx) : y[D] - mx;
    }
}

}  // namespace

void launch_margin64(const NetView& net, const QueryView* d_qs, unsigned long long t, double* d_out,
                     cudaStream_t st) {
    const size_t smem = sizeof(double) * (net.total + net.hmax);
    cudaFuncSetAttribute(k_margin64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_margin64<<<1, T64, smem, st>>>(net, d_qs, t, d_out);
}

void launch_fp64(const NetView& net, const QueryView* d_qs, int nq, const QEntry* gather,
                 const unsigned long long* gather_count, unsigned long long gather_cap,
                 unsigned long long range_lo, unsigned long long range_hi, int n_sm,
                 cudaStream_t st) {
    const size_t smem = sizeof(double) * (net.total + net.hmax) + 2 * (size_t)net.total;
    cudaFuncSetAttribute(k_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    unsigned grid = (unsigned)n_sm * 8;
    if (!gather) {
        unsigned long long n = range_hi - range_lo;
        if (n < grid) grid = (unsigned)(n ? n : 1);
    }
    k_fp64<<<grid, T64, smem, st>>>(net, d_qs, gather, gather_count, gather_cap, range_lo,
                                    range_hi);
}

}  // namespace vbmc
