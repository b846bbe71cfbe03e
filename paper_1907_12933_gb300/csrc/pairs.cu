// pairs.cu -- the covering methods of Sec. III-B over a set of input pairs
// (x1, x2) without enumeration: one CTA per pair, FP64 potentials of both
// inputs (Eq. 1, the hidden activation on layers 1..L-1), then per pair
//   sc(n)   sign change (sign(u) = 1 iff u >= 0)
//   vc(n)   no sign change and max(|u1|, |u2|) >= g min(|u1|, |u2|)
//   dc(k)   no sign change in layer k and ||u_k(x1) - u_k(x2)||_2 >= d
//   SS (i, j): i the only sign change of layer k and sc(j)      (pair bits)
//   SV (i, j): i the only sign change of layer k and vc(j)      (pair bits)
//   DS (k, j): dc(k) and sc(j)   (bit of neuron j of layer k+1; covers (any i, j))
//   DV (k, j): dc(k) and vc(j)
// ORed over all pairs into the caller's masks. Ties: a potential with |u| <
// 1e-9 in either input, a ratio test |max - g min| <= 1e-9 or a distance test
// |dist - d| <= 1e-9 is undecided; a pair that holds only under some
// resolution of the undecided tests goes to the tie mask.
#include "../../include/vbmc.h"
#include "dev.cuh"
#include "launch.h"

#include <cmath>
#include <vector>

namespace vbmc {
const NetView* net_view(const vbmc_net* net);
vbmc_status set_error(vbmc_status st, const char* msg);
}  // namespace vbmc

using namespace vbmc;

namespace {

constexpr int TP = 256;

__device__ __forceinline__ double act64p(int act, double u) {
    if (act == ACT_SIGMOID) return 1.0 / (1.0 + exp(-u));
    if (act == ACT_RELU) return u > 0.0 ? u : 0.0;
    return u;
}

struct PairOut {
    uint32_t *flip, *flip_tie, *ss, *ss_tie, *sv, *sv_tie, *ds, *ds_tie, *dv, *dv_tie;
};

// Potentials of layers l0..L into u, layer l0-1 already in u (l0 >= 2) or the
// input x (grey levels / 255, l0 = 1).
__device__ void forward64_from(const NetView& net, int l0, const uint8_t* x, double* u, double* h) {
    const int H0 = net.dims[0];
    if (l0 == 1) {
        for (int j = threadIdx.x; j < H0; j += blockDim.x) h[j] = (double)x[j] / 255.0;
        __syncthreads();
    }
    for (int l = l0; l <= net.L; ++l) {
        const int K = net.dims[l - 1], N = net.dims[l];
        const float* WT = net.WT[l];
        const double* in = l == 1 ? h : u + net.noff[l - 1];
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            double acc = (double)net.b[l][i];
            for (int j = 0; j < K; ++j) {
                const double hj = l == 1 ? in[j] : act64p(net.act, in[j]);
                acc = fma((double)WT[(size_t)j * N + i], hj, acc);
            }
            u[net.noff[l] + i] = acc;
        }
        __syncthreads();
    }
}

// Potentials of every non-input neuron for input x (grey levels / 255) into u.
__device__ void forward64(const NetView& net, const uint8_t* x, double* u, double* h) {
    forward64_from(net, 1, x, u, h);
}

// Shared scratch of one CTA: the two inputs' potentials and per-neuron flags.
struct PairScratch {
    double *u1, *u2, *h;
    unsigned char *fl, *ti, *vc, *vt;  // certain sign change, sign tie, certain value change, undecided
};

__device__ PairScratch pair_scratch(const NetView& net, double* sh) {
    const int total = net.total, H0 = net.dims[0];
    const int gw = H0 > net.hmax ? H0 : net.hmax;
    PairScratch P;
    P.u1 = sh;
    P.u2 = P.u1 + total;
    P.h = P.u2 + total;  // [gw]
    P.fl = reinterpret_cast<unsigned char*>(P.h + gw);
    P.ti = P.fl + total;
    P.vc = P.ti + total;
    P.vt = P.vc + total;
    return P;
}

// The covers of one pair from its potentials u1, u2 (all threads of the CTA).
__device__ void pair_covers(const NetView& net, const PairScratch& P, double g, double d, const PairOut& o) {
    __shared__ int nflip[kMaxL + 2], ntie[kMaxL + 2], only[kMaxL + 2];
    __shared__ double dist2[kMaxL + 2];
    const int total = net.total;
    const double tau = kTau;
    if (threadIdx.x <= kMaxL + 1) {
        nflip[threadIdx.x] = 0;
        ntie[threadIdx.x] = 0;
        only[threadIdx.x] = -1;
        dist2[threadIdx.x] = 0.0;
    }
    __syncthreads();
    for (int n = threadIdx.x; n < total; n += blockDim.x) {
        const double a1 = P.u1[n], a2 = P.u2[n];
        const bool t = fabs(a1) < tau || fabs(a2) < tau;
        const bool f = !t && ((a1 >= 0.0) != (a2 >= 0.0));
        const double a = fabs(a1), b = fabs(a2);
        const double test = fmax(a, b) - g * fmin(a, b);
        const bool v = !f && !t && test > tau;
        P.ti[n] = t;
        P.fl[n] = f;
        P.vc[n] = v;
        P.vt[n] = !f && !v && (t || fabs(test) <= tau);
        int l = 1;
        while (l < net.L && n >= net.noff[l + 1]) ++l;
        if (f) {
            atomicAdd(&nflip[l], 1);
            atomicMax(&only[l], n - net.noff[l]);
            if (o.flip) set_bit_once(o.flip, (unsigned long long)n);
        }
        if (t) {
            atomicAdd(&ntie[l], 1);
            if (o.flip_tie) set_bit_once(o.flip_tie, (unsigned long long)n);
        }
        const double e = a1 - a2;
        atomicAdd(&dist2[l], e * e);
    }
    __syncthreads();
    for (int l = 1; l < net.L; ++l) {
        const int Hl = net.dims[l], Hn = net.dims[l + 1], off = net.noff[l], on = net.noff[l + 1];
        const double dist = sqrt(dist2[l]);
        const bool dc_cert = nflip[l] == 0 && ntie[l] == 0 && dist - d > tau;
        const bool dc_poss = nflip[l] == 0 && dist - d >= -tau;
        for (int i = threadIdx.x; i < Hn; i += blockDim.x) {
            const int ni = on + i;
            const unsigned long long bit = (unsigned long long)ni;
            if (dc_cert && P.fl[ni]) { if (o.ds) set_bit_once(o.ds, bit); }
            else if (dc_poss && (P.fl[ni] || P.ti[ni])) { if (o.ds_tie) set_bit_once(o.ds_tie, bit); }
            if (dc_cert && P.vc[ni]) { if (o.dv) set_bit_once(o.dv, bit); }
            else if (dc_poss && (P.vc[ni] || P.vt[ni])) { if (o.dv_tie) set_bit_once(o.dv_tie, bit); }
        }
        // SS and SV: j the only changed neuron of layer l (for certain, or under ties)
        const int nf = nflip[l], nt = ntie[l], oj = only[l];
        for (int e = threadIdx.x; e < Hl * Hn; e += blockDim.x) {
            const int j = e / Hn, i = e % Hn;
            const bool certain = nt == 0 && nf == 1 && j == oj;
            const bool possible = certain || (nt > 0 && ((nf == 1 && j == oj) || (nf == 0 && P.ti[off + j])));
            if (!possible) continue;
            const int ni = on + i;
            const unsigned long long bit = (unsigned long long)net.ssoff[l] + (unsigned long long)j * Hn + i;
            if (certain && P.fl[ni]) { if (o.ss) set_bit_once(o.ss, bit); }
            else if (P.fl[ni] || P.ti[ni]) { if (o.ss_tie) set_bit_once(o.ss_tie, bit); }
            if (certain && P.vc[ni]) { if (o.sv) set_bit_once(o.sv, bit); }
            else if (P.vc[ni] || P.vt[ni]) { if (o.sv_tie) set_bit_once(o.sv_tie, bit); }
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(TP) k_pairs(NetView net, const uint8_t* x1s, const uint8_t* x2s, int n_pairs,
                                               double g, double d, PairOut o) {
    extern __shared__ double sh[];
    const PairScratch P = pair_scratch(net, sh);
    const int H0 = net.dims[0];
    for (int p = blockIdx.x; p < n_pairs; p += gridDim.x) {
        forward64(net, x1s + (size_t)p * H0, P.u1, P.h);
        forward64(net, x2s + (size_t)p * H0, P.u2, P.h);
        pair_covers(net, P, g, d, o);
    }
}

// The covers over the enumeration: the pairs (x, x_t) of the unperturbed image
// and each point t of [lo, hi) that passes the query's filter. x's potentials
// once per CTA; x_t's layer 1 incrementally from them (its s changed pixels),
// layers 2..L in full.
__global__ void __launch_bounds__(TP) k_enum_pairs(NetView net, QueryView Q, double g, double d, PairOut o,
                                                    unsigned long long* n_points) {
    extern __shared__ double sh[];
    const PairScratch P = pair_scratch(net, sh);
    __shared__ int dv[kMaxS];
    __shared__ int pass;
    const int H1 = net.dims[1];
    forward64(net, Q.image, P.u1, P.h);
    unsigned long long mine = 0;
    for (unsigned long long t = Q.lo + blockIdx.x; t < Q.hi; t += gridDim.x) {
        if (threadIdx.x == 0) {
            int dg[kMaxS];
            decode_digits(t, Q.s, Q.R, dg);
            long long s2 = 0;
            bool shell = Q.k == 0;
            for (int p = 0; p < Q.s; ++p) {
                const int v0 = Q.image[Q.pix_in[p]];
                int v1 = v0 + dg[p] - Q.k;
                v1 = v1 < 0 ? 0 : (v1 > 255 ? 255 : v1);
                dv[p] = v1 - v0;
                s2 += (long long)dv[p] * dv[p];
                shell = shell || dg[p] == 0 || dg[p] == Q.R - 1;
            }
            // the query's filter (the Euclidean ball of Eq. 9 on the grid, a k-shell)
            pass = (!(Q.filter & FILTER_L2) || s2 <= Q.l2max) && (!(Q.filter & FILTER_SHELL) || shell);
        }
        __syncthreads();
        if (!pass) {
            __syncthreads();
            continue;
        }
        ++mine;
        for (int j = threadIdx.x; j < H1; j += blockDim.x) {
            double a = P.u1[j];
            for (int p = 0; p < Q.s; ++p)
                a = fma((double)net.WT[1][(size_t)Q.pix_in[p] * H1 + j], (double)dv[p] / 255.0, a);
            P.u2[j] = a;
        }
        __syncthreads();
        forward64_from(net, 2, nullptr, P.u2, P.h);
        pair_covers(net, P, g, d, o);
    }
    if (threadIdx.x == 0 && mine) atomicAdd(n_points, mine);
}

}  // namespace

namespace vbmc {

// Clears the caller's masks and checks the cover parameters and the kernels'
// shared-memory need; sets *smem.
vbmc_status pair_setup(const NetView& v, const vbmc_cover_params* params, const vbmc_pair_masks* out,
                       cudaStream_t st, size_t* smem) {
    if (!(params->g >= 1.0) || !(params->d >= 0.0)) return set_error(VBMC_ERR_ARG, "need g >= 1 and d >= 0");
    const size_t fw = (size_t)v.flip_words * 4, sw = (size_t)v.ss_words * 4;
    uint32_t* const fmasks[6] = {out->flip, out->flip_tie, out->ds, out->ds_tie, out->dv, out->dv_tie};
    uint32_t* const smasks[4] = {out->ss, out->ss_tie, out->sv, out->sv_tie};
    for (uint32_t* m : fmasks)
        if (m && cudaMemsetAsync(m, 0, fw, st) != cudaSuccess) return set_error(VBMC_ERR_CUDA, "memset");
    for (uint32_t* m : smasks)
        if (m && sw && cudaMemsetAsync(m, 0, sw, st) != cudaSuccess) return set_error(VBMC_ERR_CUDA, "memset");
    const int gw = v.dims[0] > v.hmax ? v.dims[0] : v.hmax;
    *smem = sizeof(double) * (2 * (size_t)v.total + gw) + 4 * (size_t)v.total;
    if (*smem > 200 * 1024) return set_error(VBMC_ERR_UNSUPPORTED, "net too large for the pair kernel");
    return VBMC_OK;
}

int pair_grid(unsigned long long units) {
    int n_sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned long long cap = (unsigned long long)n_sm * 4;
    return (int)(units < cap ? units : cap);
}

// The covers over the pairs (unperturbed image, point) of the view's range;
// adds the points that pass the filter to *d_npoints.
vbmc_status launch_enum_pairs(const NetView& v, const QueryView& q, const vbmc_cover_params* params,
                              const vbmc_pair_masks* out, unsigned long long* d_npoints, cudaStream_t st) {
    size_t smem = 0;
    vbmc_status s = pair_setup(v, params, out, st, &smem);
    if (s != VBMC_OK) return s;
    if (q.hi <= q.lo) return VBMC_OK;
    cudaFuncSetAttribute(k_enum_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const PairOut o{out->flip, out->flip_tie, out->ss, out->ss_tie, out->sv, out->sv_tie,
                    out->ds, out->ds_tie, out->dv, out->dv_tie};
    k_enum_pairs<<<pair_grid(q.hi - q.lo), TP, smem, st>>>(v, q, params->g, params->d, o, d_npoints);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VBMC_OK : set_error(VBMC_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace vbmc

extern "C" vbmc_status vbmc_pair_coverage(const vbmc_net* net, const uint8_t* d_images1, const uint8_t* d_images2,
                                          int32_t n_pairs, const vbmc_cover_params* params,
                                          const vbmc_pair_masks* out, void* stream) {
    if (!net || !params || !out || (n_pairs > 0 && (!d_images1 || !d_images2)))
        return set_error(VBMC_ERR_ARG, "null argument");
    if (n_pairs < 0) return set_error(VBMC_ERR_ARG, "n_pairs must be >= 0");
    const NetView& v = *net_view(net);
    cudaStream_t st = (cudaStream_t)stream;
    size_t smem = 0;
    vbmc_status s = pair_setup(v, params, out, st, &smem);
    if (s != VBMC_OK || n_pairs == 0) return s;
    cudaFuncSetAttribute(k_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const PairOut o{out->flip, out->flip_tie, out->ss, out->ss_tie, out->sv, out->sv_tie,
                    out->ds, out->ds_tie, out->dv, out->dv_tie};
    k_pairs<<<pair_grid((unsigned long long)n_pairs), TP, smem, st>>>(v, d_images1, d_images2, n_pairs, params->g,
                                                                    params->d, o);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VBMC_OK : set_error(VBMC_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" vbmc_status vbmc_covered_fraction(const vbmc_net* net, int32_t layout, const uint32_t* mask,
                                             double* fraction) {
    if (!net || !mask || !fraction) return set_error(VBMC_ERR_ARG, "null argument");
    if (layout != VBMC_LAYOUT_PAIRS && layout != VBMC_LAYOUT_LAYER)
        return set_error(VBMC_ERR_ARG, "layout must be VBMC_LAYOUT_PAIRS or VBMC_LAYOUT_LAYER");
    const NetView& v = *net_view(net);
    std::vector<char> cov((size_t)v.total, 0);
    auto bit = [&](unsigned long long b) { return (mask[b >> 5] >> (b & 31)) & 1u; };
    for (int l = 1; l < v.L; ++l) {
        const int Hl = v.dims[l], Hn = v.dims[l + 1], off = v.noff[l], on = v.noff[l + 1];
        if (layout == VBMC_LAYOUT_PAIRS) {
            for (int j = 0; j < Hl; ++j)
                for (int i = 0; i < Hn; ++i)
                    if (bit((unsigned long long)v.ssoff[l] + (unsigned long long)j * Hn + i)) {
                        cov[off + j] = 1;
                        cov[on + i] = 1;
                    }
        } else {
            for (int i = 0; i < Hn; ++i)
                if (bit((unsigned long long)(on + i))) {
                    cov[on + i] = 1;
                    for (int j = 0; j < Hl; ++j) cov[off + j] = 1;
                }
        }
    }
    long c = 0;
    for (char x : cov) c += x;
    *fraction = v.total ? (double)c / (double)v.total : 0.0;
    return VBMC_OK;
}
