// proposal.cu -- learned tile proposal: a small MLP that ranks contiguous
// tiles of a query's index space so that a point violating Eq. 10 (a witness)
// is met sooner when the tiles are checked in its order. A SAFE verdict still
// needs every tile, so the order never changes a verdict, only the time to the
// first witness.
//
// Features of a query, 3 x H_0 (input of the proposal net):
//   x_j      the unperturbed image, grey level / 255
//   m_j      R^-p at the p-th listed pixel (its digit's place value in the
//            point index relative to the leading digit), 0 elsewhere
//   g_j      m_j * dM/dx_j * (k / 255) / max(M, eps): the input gradient of
//            the margin M = y_D - y_r at the unperturbed image (r: runner-up
//            class), through the verified net's ReLU layers, as the fraction
//            of the margin one full step of pixel j would use up to first
//            order; clipped to [-kFeatClip, kFeatClip]
// The tile index is led by the first pixel's digit, so the place-value
// weights make sum_j g_j track the quantity that decides which tiles reach
// the decision boundary first, for every pixel position.
//
// The proposal net F -> H1 -> H2 -> T (ReLU hidden layers) scores the T tiles.
// Training objective (listwise softmax cross-entropy): with p = softmax(z)
// and t the 0/1 witness labels of a query's tiles,
//   loss = -sum_i (t_i / sum t) log p_i,   dL/dz = p - t / sum t,
// averaged over the queries that have at least one witness tile (the others
// carry no weight). The optimiser is Adam with decoupled weight decay.
// Forward and backward run in FP32 on CUDA cores; the training forward and
// the inference forward round weights and activations to BF16 first (FP32
// accumulation), the precision the proposal net runs in.
#include "../../include/vbmc.h"
#include "dev.cuh"
#include "launch.h"

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

namespace vbmc {
const NetView* net_view(const vbmc_net* net);
vbmc_status set_error(vbmc_status st, const char* msg);
}  // namespace vbmc

using namespace vbmc;

struct vbmc_proposal {
    int dims[4];              // F, H1, H2, T
    float* W[4] = {};         // W[l]: dims[l] x dims[l-1] row-major, l = 1..3
    float* b[4] = {};
    float* mW[4] = {};        // Adam moments
    float* vW[4] = {};
    float* mb[4] = {};
    float* vb[4] = {};
    float* gW[4] = {};        // gradients of the last vbmc_proposal_grads call
    float* gb[4] = {};
    float* act[4] = {};       // activations of the last forward (act[0]: input copy)
    float* dact[4] = {};
    float* loss = nullptr;    // [2]: loss sum, number of weighted rows
    int bmax = 0;
    long step = 0;
    std::vector<void*> owned;
};

namespace {

constexpr float kFeatClip = 16.f;
constexpr int GT = 64;   // GEMM tile (rows and columns)
constexpr int GK = 16;   // GEMM k step

__device__ __forceinline__ float rnd_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// C[M][N] = sum_k A(m, k) B(k, n) (+ bias[n]) (ReLU) (masked by mask[m][n] > 0)
//   A(m, k) = TA ? A[k * lda + m] : A[m * lda + k]
//   B(k, n) = TB ? B[n * ldb + k] : B[k * ldb + n]
// 64 x 64 tile per CTA of 256 threads, 4 x 4 outputs per thread; bf != 0
// rounds both operands to BF16 as they are staged.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                              const float* __restrict__ B, int ldb, float* __restrict__ C,
                                              int ldc, const float* __restrict__ bias,
                                              const float* __restrict__ mask, int relu, int bf) {
    __shared__ float As[GK][GT + 4];
    __shared__ float Bs[GK][GT + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + r * 256;
            int m, k;
            if (TA) { k = e / GT; m = e % GT; } else { m = e / GK; k = e % GK; }
            const int gm = m0 + m, gk = k0 + k;
            float a = 0.f;
            if (gm < M && gk < K) a = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
            As[k][m] = bf ? rnd_bf16(a) : a;
            int n, kb;
            if (TB) { n = e / GK; kb = e % GK; } else { kb = e / GT; n = e % GT; }
            const int gn = n0 + n, gkb = k0 + kb;
            float bv = 0.f;
            if (gn < N && gkb < K) bv = TB ? B[(size_t)gn * ldb + gkb] : B[(size_t)gkb * ldb + gn];
            Bs[kb][n] = bf ? rnd_bf16(bv) : bv;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float v = acc[i][j];
            if (bias) v += bias[n];
            if (relu) v = fmaxf(v, 0.f);
            if (mask && !(mask[(size_t)m * ldc + n] > 0.f)) v = 0.f;
            C[(size_t)m * ldc + n] = v;
        }
    }
}

template <bool TA, bool TB>
void gemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
          const float* bias, const float* mask, int relu, int bf, cudaStream_t st) {
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
    k_gemm<TA, TB><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, mask, relu, bf);
}

// Column sums: out[n] = sum_m X[m][n] (bias gradients).
__global__ void k_colsum(const float* X, int M, int N, float* out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float acc = 0.f;
    for (int m = 0; m < M; ++m) acc += X[(size_t)m * N + n];
    out[n] = acc;
}

// Listwise softmax cross-entropy, one warp per row: dZ = p - t / sum t
// (0 for rows without a witness tile), loss[0] += row loss, loss[1] += 1.
__global__ void k_softmax_ce(const float* Z, const float* Tg, float* dZ, float* loss, int B, int T) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= B) return;
    const float* z = Z + (size_t)warp * T;
    const float* t = Tg + (size_t)warp * T;
    float mx = -INFINITY, ts = 0.f;
    for (int i = lane; i < T; i += 32) {
        mx = fmaxf(mx, z[i]);
        ts += t[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        ts += __shfl_xor_sync(0xffffffffu, ts, o);
    }
    float se = 0.f;
    for (int i = lane; i < T; i += 32) se += expf(z[i] - mx);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    const float lse = mx + logf(se);
    float l = 0.f;
    for (int i = lane; i < T; i += 32) {
        const float q = ts > 0.f ? t[i] / ts : 0.f;
        dZ[(size_t)warp * T + i] = ts > 0.f ? expf(z[i] - lse) - q : 0.f;
        l -= q * (z[i] - lse);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (lane == 0 && ts > 0.f) {
        atomicAdd(&loss[0], l);
        atomicAdd(&loss[1], 1.f);
    }
}

// dZ /= number of weighted rows (the loss is their mean).
__global__ void k_scale_by_count(float* dZ, long n, const float* loss) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float c = loss[1];
    dZ[i] = c > 0.f ? dZ[i] / c : 0.f;
}

// Adam with decoupled weight decay (bias-corrected moments).
__global__ void k_adamw(float* w, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                        float eps, float c1, float c2, float wd) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * w[i]);
}

// Features of one query per CTA (see the file header). Shared memory: the
// potentials of every layer, two gradient buffers of max(H_0, hmax) floats.
__global__ void k_features(NetView net, const uint8_t* images, const int* pixels, const int* s_of,
                           const int* k_of, int pix_stride, float* F, float* reach, float* margin) {
    extern __shared__ float sh[];
    const int q = blockIdx.x;
    const int H0 = net.dims[0], L = net.L;
    const int gw = H0 > net.hmax ? H0 : net.hmax;
    const uint8_t* img = images + (size_t)q * H0;
    const int* pix = pixels + (size_t)q * pix_stride;
    const int s = min(max(s_of[q], 0), pix_stride), k = max(k_of[q], 0);
    float* u = sh;              // [total]
    float* g = u + net.total;   // [gw]
    float* g2 = g + gw;         // [gw]
    float* out = F + (size_t)q * 3 * H0;
    for (int j = threadIdx.x; j < H0; j += blockDim.x) {
        g2[j] = (float)img[j] / 255.f;  // the input, kept in g2 during the forward pass
        out[j] = g2[j];
        out[H0 + j] = 0.f;
        out[2 * H0 + j] = 0.f;
    }
    __syncthreads();
    // forward: u_l = W_l h_{l-1} + b_l (Eq. 1), h = ReLU(u) on hidden layers
    for (int l = 1; l <= L; ++l) {
        const int K = net.dims[l - 1], N = net.dims[l];
        const float* WT = net.WT[l];
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            float acc = net.b[l][i];
            for (int j = 0; j < K; ++j) {
                const float h = l == 1 ? g2[j] : fmaxf(u[net.noff[l - 1] + j], 0.f);
                acc = fmaf(WT[(size_t)j * N + i], h, acc);
            }
            u[net.noff[l] + i] = acc;
        }
        __syncthreads();
    }
    const int HL = net.dims[L];
    const float* y = u + net.noff[L];
    int D = 0;
    for (int i = 1; i < HL; ++i)
        if (y[i] > y[D]) D = i;
    int r = D == 0 ? 1 : 0;
    for (int i = 0; i < HL; ++i)
        if (i != D && y[i] > y[r]) r = i;
    const float M = y[D] - y[r];
    for (int i = threadIdx.x; i < HL; i += blockDim.x) g[i] = (i == D) ? 1.f : (i == r ? -1.f : 0.f);
    __syncthreads();
    // backward: dM/dh_{l-1} = W_l^T dM/du_l, times ReLU'(u_{l-1}) on hidden layers
    for (int l = L; l >= 1; --l) {
        const int K = net.dims[l - 1], N = net.dims[l];
        const float* W = net.W[l];
        for (int j = threadIdx.x; j < K; j += blockDim.x) {
            float acc = 0.f;
            for (int i = 0; i < N; ++i) acc = fmaf(W[(size_t)i * K + j], g[i], acc);
            if (l > 1 && !(u[net.noff[l - 1] + j] > 0.f)) acc = 0.f;
            g2[j] = acc;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < K; j += blockDim.x) g[j] = g2[j];
        __syncthreads();
    }
    const int R = 2 * k + 1;
    const float scale = ((float)k / 255.f) / fmaxf(M, 1e-6f);
    if (threadIdx.x == 0) {
        float pv = 1.f, rs = 0.f;
        for (int p = 0; p < s; ++p) {
            const int j = pix[p];
            if (j < 0 || j >= H0) continue;  // the verify calls reject such lists
            const float e = g[j] * scale;
            out[H0 + j] = pv;
            out[2 * H0 + j] = fminf(kFeatClip, fmaxf(-kFeatClip, pv * e));
            rs += fabsf(e);
            pv /= (float)R;
        }
        if (reach) reach[q] = rs;
        if (margin) margin[q] = M;
    }
}

// Tile order of each query: order[q][rank] = tile, by descending score, lower
// tile index first on equal scores. One CTA per query, one thread per tile.
__global__ void k_rank(const float* scores, int T, int* order) {
    const int q = blockIdx.x;
    const float* z = scores + (size_t)q * T;
    for (int i = threadIdx.x; i < T; i += blockDim.x) {
        const float zi = z[i];
        int rank = 0;
        for (int j = 0; j < T; ++j) rank += (z[j] > zi) || (z[j] == zi && j < i);
        order[(size_t)q * T + rank] = i;
    }
}

// Adversarial points per tile from a verdict bitmap: tile i covers
// [i * tsize, min((i + 1) * tsize, n)). One CTA per tile.
__global__ void k_tile_counts(const uint32_t* bitmap, unsigned long long n, unsigned long long tsize,
                              unsigned long long* counts) {
    const unsigned long long a = (unsigned long long)blockIdx.x * tsize;
    const unsigned long long b = a + tsize < n ? a + tsize : n;
    unsigned long long c = 0;
    if (a < b) {
        for (unsigned long long w = a / 32 + threadIdx.x; w <= (b - 1) / 32; w += blockDim.x) {
            uint32_t x = bitmap[w];
            const unsigned long long base = w * 32;
            if (base < a) x &= ~0u << (unsigned)(a - base);
            if (base + 32 > b) x &= (1u << (unsigned)(b - base)) - 1u;  // b - base in [1, 31]
            c += __popc(x);
        }
    }
    __shared__ unsigned long long part[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        counts[blockIdx.x] = t;
    }
}

unsigned nblk(long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

namespace vbmc {

void launch_tile_counts(const uint32_t* d_bitmap, unsigned long long n, int n_tiles,
                        unsigned long long* d_counts, cudaStream_t st) {
    const unsigned long long tsize = (n + n_tiles - 1) / n_tiles;
    k_tile_counts<<<n_tiles, 256, 0, st>>>(d_bitmap, n, tsize ? tsize : 1, d_counts);
}

}  // namespace vbmc

extern "C" vbmc_status vbmc_proposal_create(int32_t n_features, int32_t h1, int32_t h2, int32_t n_tiles,
                                            int32_t max_batch, uint64_t seed, vbmc_proposal** out) {
    if (!out || n_features < 1 || h1 < 1 || h2 < 1 || n_tiles < 2 || n_tiles > 1024 || max_batch < 1)
        return set_error(VBMC_ERR_ARG, "bad proposal shape");
    vbmc_proposal* p = new vbmc_proposal();
    p->dims[0] = n_features;
    p->dims[1] = h1;
    p->dims[2] = h2;
    p->dims[3] = n_tiles;
    p->bmax = max_batch;
    cudaError_t e = cudaSuccess;
    auto A = [&](float** ptr, size_t n) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(ptr, sizeof(float) * (n ? n : 1));
        if (e == cudaSuccess) {
            p->owned.push_back(*ptr);
            e = cudaMemset(*ptr, 0, sizeof(float) * (n ? n : 1));
        }
    };
    // He-normal weights, zero biases: SplitMix64 counter stream, Box-Muller
    auto mix = [](uint64_t z) {
        z ^= z >> 30;
        z *= 0xBF58476D1CE4E5B9ull;
        z ^= z >> 27;
        z *= 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    uint64_t ctr = mix(seed ^ 0x6A09E667F3BCC908ull);
    for (int l = 1; l <= 3; ++l) {
        const size_t n = (size_t)p->dims[l] * p->dims[l - 1];
        A(&p->W[l], n);
        A(&p->b[l], p->dims[l]);
        A(&p->mW[l], n);
        A(&p->vW[l], n);
        A(&p->mb[l], p->dims[l]);
        A(&p->vb[l], p->dims[l]);
        A(&p->gW[l], n);
        A(&p->gb[l], p->dims[l]);
        std::vector<float> h(n);
        const double sd = std::sqrt(2.0 / p->dims[l - 1]);
        for (size_t i = 0; i < n; ++i) {
            ctr += 0x9E3779B97F4A7C15ull;
            const double u1 = ((mix(ctr) >> 11) + 1.0) * 0x1p-53;
            ctr += 0x9E3779B97F4A7C15ull;
            const double u2 = (mix(ctr) >> 11) * 0x1p-53;
            h[i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
        if (e == cudaSuccess) e = cudaMemcpy(p->W[l], h.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    }
    for (int l = 0; l <= 3; ++l) {
        A(&p->act[l], (size_t)max_batch * p->dims[l]);
        A(&p->dact[l], (size_t)max_batch * p->dims[l]);
    }
    A(&p->loss, 2);
    if (e != cudaSuccess) {
        vbmc_proposal_free(p);
        return set_error(VBMC_ERR_OOM, "proposal_create: device allocation failed");
    }
    *out = p;
    return VBMC_OK;
}

extern "C" vbmc_status vbmc_proposal_free(vbmc_proposal* p) {
    if (!p) return VBMC_OK;
    cudaDeviceSynchronize();
    for (void* x : p->owned) cudaFree(x);
    delete p;
    return VBMC_OK;
}

namespace {

// act[0] = X; act[l] = act_l(W_l act[l-1] + b_l), l = 1..3 (ReLU on 1, 2).
void forward(vbmc_proposal* p, const float* d_X, int B, int bf, cudaStream_t st) {
    cudaMemcpyAsync(p->act[0], d_X, sizeof(float) * (size_t)B * p->dims[0], cudaMemcpyDeviceToDevice, st);
    for (int l = 1; l <= 3; ++l) {
        const int K = p->dims[l - 1], N = p->dims[l];
        gemm<false, true>(B, N, K, p->act[l - 1], K, p->W[l], K, p->act[l], N, p->b[l], nullptr, l < 3, bf,
                          st);
    }
}

vbmc_status check_batch(const vbmc_proposal* p, const void* a, const void* b, int B) {
    if (!p || !a || !b) return set_error(VBMC_ERR_ARG, "null argument");
    if (B < 1 || B > p->bmax) return set_error(VBMC_ERR_ARG, "batch size outside [1, max_batch]");
    return VBMC_OK;
}

}  // namespace

extern "C" vbmc_status vbmc_proposal_scores(vbmc_proposal* p, const float* d_X, int32_t B, float* d_scores,
                                            int32_t* d_order, void* stream) {
    vbmc_status s = check_batch(p, d_X, d_scores, B);
    if (s != VBMC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    forward(p, d_X, B, 1, st);
    cudaMemcpyAsync(d_scores, p->act[3], sizeof(float) * (size_t)B * p->dims[3], cudaMemcpyDeviceToDevice, st);
    if (d_order) k_rank<<<B, 256, 0, st>>>(p->act[3], p->dims[3], d_order);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VBMC_OK : set_error(VBMC_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" vbmc_status vbmc_proposal_grads(vbmc_proposal* p, const float* d_X, const float* d_T, int32_t B,
                                           int32_t bf16, float* h_loss, void* stream) {
    vbmc_status s = check_batch(p, d_X, d_T, B);
    if (s != VBMC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    forward(p, d_X, B, bf16 ? 1 : 0, st);
    cudaMemsetAsync(p->loss, 0, sizeof(float) * 2, st);
    const int T = p->dims[3];
    k_softmax_ce<<<nblk((long)B * 32, 256), 256, 0, st>>>(p->act[3], d_T, p->dact[3], p->loss, B, T);
    k_scale_by_count<<<nblk((long)B * T, 256), 256, 0, st>>>(p->dact[3], (long)B * T, p->loss);
    for (int l = 3; l >= 1; --l) {
        const int K = p->dims[l - 1], N = p->dims[l];
        // dW_l = dact_l^T act_{l-1}   (N x K),  db_l = column sums of dact_l
        gemm<true, false>(N, K, B, p->dact[l], N, p->act[l - 1], K, p->gW[l], K, nullptr, nullptr, 0, 0, st);
        k_colsum<<<nblk(N, 256), 256, 0, st>>>(p->dact[l], B, N, p->gb[l]);
        // dact_{l-1} = (dact_l W_l) * ReLU'(act_{l-1})
        if (l > 1)
            gemm<false, false>(B, K, N, p->dact[l], N, p->W[l], K, p->dact[l - 1], K, nullptr, p->act[l - 1], 0,
                               0, st);
    }
    if (h_loss) {
        float hl[2];
        cudaMemcpyAsync(hl, p->loss, sizeof(hl), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        *h_loss = hl[1] > 0.f ? hl[0] / hl[1] : 0.f;
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VBMC_OK : set_error(VBMC_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" vbmc_status vbmc_proposal_train_step(vbmc_proposal* p, const float* d_X, const float* d_T,
                                                int32_t B, float lr, float weight_decay, float* h_loss,
                                                void* stream) {
    vbmc_status s = vbmc_proposal_grads(p, d_X, d_T, B, 1, h_loss, stream);
    if (s != VBMC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    p->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - std::pow(b1, (float)p->step), c2 = 1.f - std::pow(b2, (float)p->step);
    for (int l = 1; l <= 3; ++l) {
        const int n = p->dims[l] * p->dims[l - 1];
        k_adamw<<<nblk(n, 256), 256, 0, st>>>(p->W[l], p->gW[l], p->mW[l], p->vW[l], n, lr, b1, b2, eps, c1, c2,
                                             weight_decay);
        k_adamw<<<nblk(p->dims[l], 256), 256, 0, st>>>(p->b[l], p->gb[l], p->mb[l], p->vb[l], p->dims[l], lr, b1,
                                                      b2, eps, c1, c2, 0.f);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VBMC_OK : set_error(VBMC_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" vbmc_status vbmc_proposal_params(vbmc_proposal* p, int32_t layer, float* h_W, float* h_b,
                                            float* h_gW, float* h_gb) {
    if (!p || layer < 1 || layer > 3) return set_error(VBMC_ERR_ARG, "layer must be 1..3");
    const size_t n = (size_t)p->dims[layer] * p->dims[layer - 1];
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && h_W) e = cudaMemcpy(h_W, p->W[layer], sizeof(float) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_b)
        e = cudaMemcpy(h_b, p->b[layer], sizeof(float) * p->dims[layer], cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_gW) e = cudaMemcpy(h_gW, p->gW[layer], sizeof(float) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_gb)
        e = cudaMemcpy(h_gb, p->gb[layer], sizeof(float) * p->dims[layer], cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? VBMC_OK : set_error(VBMC_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" vbmc_status vbmc_proposal_set_params(vbmc_proposal* p, int32_t layer, const float* h_W,
                                                const float* h_b) {
    if (!p || layer < 1 || layer > 3) return set_error(VBMC_ERR_ARG, "layer must be 1..3");
    const size_t n = (size_t)p->dims[layer] * p->dims[layer - 1];
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && h_W) e = cudaMemcpy(p->W[layer], h_W, sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && h_b)
        e = cudaMemcpy(p->b[layer], h_b, sizeof(float) * p->dims[layer], cudaMemcpyHostToDevice);
    return e == cudaSuccess ? VBMC_OK : set_error(VBMC_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" vbmc_status vbmc_proposal_features(const vbmc_net* net, const uint8_t* d_images,
                                              const int32_t* d_pixels, const int32_t* d_s, const int32_t* d_k,
                                              int32_t pix_stride, int32_t nq, float* d_features,
                                              float* d_reach, float* d_margin, void* stream) {
    if (!net || !d_images || !d_pixels || !d_s || !d_k || !d_features || nq < 1 || pix_stride < 0)
        return set_error(VBMC_ERR_ARG, "null argument or empty batch");
    const NetView& v = *net_view(net);
    if (v.act != ACT_RELU) return set_error(VBMC_ERR_UNSUPPORTED, "features need a ReLU net");
    const int gw = v.dims[0] > v.hmax ? v.dims[0] : v.hmax;
    const size_t smem = sizeof(float) * (v.total + 2 * (size_t)gw);
    if (smem > 200 * 1024) return set_error(VBMC_ERR_UNSUPPORTED, "net too large for the feature kernel");
    cudaFuncSetAttribute(k_features, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_features<<<nq, 256, smem, (cudaStream_t)stream>>>(v, d_images, d_pixels, d_s, d_k, pix_stride, d_features,
                                                       d_reach, d_margin);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VBMC_OK : set_error(VBMC_ERR_CUDA, cudaGetErrorString(e));
}
