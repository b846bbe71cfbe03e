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

// Potentials of every non-input neuron for input x (grey levels / 255) into u.
__device__ void forward64(const NetView& net, const uint8_t* x, double* u, double* h) {
    const int H0 = net.dims[0];
    for (int j = threadIdx.x; j < H0; j += blockDim.x) h[j] = (double)x[j] / 255.0;
    __syncthreads();
    for (int l = 1; l <= net.L; ++l) {
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

__global__ void __launch_bounds__(TP) k_pairs(NetView net, const uint8_t* x1s, const uint8_t* x2s, int n_pairs,
                                               double g, double d, PairOut o) {
    extern __shared__ double sh[];
    const int total = net.total, H0 = net.dims[0];
    const int gw = H0 > net.hmax ? H0 : net.hmax;
    double* u1 = sh;
    double* u2 = u1 + total;
    double* h = u2 + total;                                                  // [gw]
    unsigned char* fl = reinterpret_cast<unsigned char*>(h + gw);            // certain sign change
    unsigned char* ti = fl + total;                                          // sign tie
    unsigned char* vc = ti + total;                                          // certain value change
    unsigned char* vt = vc + total;                                          // value change undecided
    __shared__ int nflip[kMaxL + 2], ntie[kMaxL + 2], only[kMaxL + 2];
    __shared__ double dist2[kMaxL + 2];
    const double tau = kTau;
    for (int p = blockIdx.x; p < n_pairs; p += gridDim.x) {
        forward64(net, x1s + (size_t)p * H0, u1, h);
        forward64(net, x2s + (size_t)p * H0, u2, h);
        if (threadIdx.x <= kMaxL + 1) {
            nflip[threadIdx.x] = 0;
            ntie[threadIdx.x] = 0;
            only[threadIdx.x] = -1;
            dist2[threadIdx.x] = 0.0;
        }
        __syncthreads();
        for (int n = threadIdx.x; n < total; n += blockDim.x) {
            const double a1 = u1[n], a2 = u2[n];
            const bool t = fabs(a1) < tau || fabs(a2) < tau;
            const bool f = !t && ((a1 >= 0.0) != (a2 >= 0.0));
            const double a = fabs(a1), b = fabs(a2);
            const double test = fmax(a, b) - g * fmin(a, b);
            const bool v = !f && !t && test > tau;
            ti[n] = t;
            fl[n] = f;
            vc[n] = v;
            vt[n] = !f && !v && (t || fabs(test) <= tau);
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
                if (dc_cert && fl[ni]) { if (o.ds) set_bit_once(o.ds, bit); }
                else if (dc_poss && (fl[ni] || ti[ni])) { if (o.ds_tie) set_bit_once(o.ds_tie, bit); }
                if (dc_cert && vc[ni]) { if (o.dv) set_bit_once(o.dv, bit); }
                else if (dc_poss && (vc[ni] || vt[ni])) { if (o.dv_tie) set_bit_once(o.dv_tie, bit); }
            }
            // SS and SV: j the only changed neuron of layer l (for certain, or under ties)
            const int nf = nflip[l], nt = ntie[l], oj = only[l];
            for (int e = threadIdx.x; e < Hl * Hn; e += blockDim.x) {
                const int j = e / Hn, i = e % Hn;
                const bool certain = nt == 0 && nf == 1 && j == oj;
                const bool possible = certain || (nt > 0 && ((nf == 1 && j == oj) || (nf == 0 && ti[off + j])));
                if (!possible) continue;
                const int ni = on + i;
                const unsigned long long bit = (unsigned long long)net.ssoff[l] + (unsigned long long)j * Hn + i;
                if (certain && fl[ni]) { if (o.ss) set_bit_once(o.ss, bit); }
                else if (fl[ni] || ti[ni]) { if (o.ss_tie) set_bit_once(o.ss_tie, bit); }
                if (certain && vc[ni]) { if (o.sv) set_bit_once(o.sv, bit); }
                else if (vc[ni] || vt[ni]) { if (o.sv_tie) set_bit_once(o.sv_tie, bit); }
            }
        }
        __syncthreads();
    }
}

}  // namespace

extern "C" vbmc_status vbmc_pair_coverage(const vbmc_net* net, const uint8_t* d_images1, const uint8_t* d_images2,
                                          int32_t n_pairs, const vbmc_cover_params* params,
                                          const vbmc_pair_masks* out, void* stream) {
    if (!net || !params || !out || (n_pairs > 0 && (!d_images1 || !d_images2)))
        return set_error(VBMC_ERR_ARG, "null argument");
    if (n_pairs < 0) return set_error(VBMC_ERR_ARG, "n_pairs must be >= 0");
    if (!(params->g >= 1.0) || !(params->d >= 0.0)) return set_error(VBMC_ERR_ARG, "need g >= 1 and d >= 0");
    const NetView& v = *net_view(net);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t fw = (size_t)v.flip_words * 4, sw = (size_t)v.ss_words * 4;
    uint32_t* const fmasks[6] = {out->flip, out->flip_tie, out->ds, out->ds_tie, out->dv, out->dv_tie};
    uint32_t* const smasks[4] = {out->ss, out->ss_tie, out->sv, out->sv_tie};
    for (uint32_t* m : fmasks)
        if (m && cudaMemsetAsync(m, 0, fw, st) != cudaSuccess) return set_error(VBMC_ERR_CUDA, "memset");
    for (uint32_t* m : smasks)
        if (m && sw && cudaMemsetAsync(m, 0, sw, st) != cudaSuccess) return set_error(VBMC_ERR_CUDA, "memset");
    if (n_pairs == 0) return VBMC_OK;
    const int gw = v.dims[0] > v.hmax ? v.dims[0] : v.hmax;
    const size_t smem = sizeof(double) * (2 * (size_t)v.total + gw) + 4 * (size_t)v.total;
    if (smem > 200 * 1024) return set_error(VBMC_ERR_UNSUPPORTED, "net too large for the pair kernel");
    cudaFuncSetAttribute(k_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n_sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = n_pairs < n_sm * 4 ? n_pairs : n_sm * 4;
    PairOut o{out->flip, out->flip_tie, out->ss, out->ss_tie, out->sv, out->sv_tie,
              out->ds, out->ds_tie, out->dv, out->dv_tie};
    k_pairs<<<grid, TP, smem, st>>>(v, d_images1, d_images2, n_pairs, params->g, params->d, o);
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
