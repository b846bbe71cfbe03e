// spectral.cu -- rigorous upper bounds of matrix spectral norms (net set-up).
//
// For a real matrix A, sigma_max(A)^2 = lambda_max(G) with G = A A^T (or A^T A),
// and for symmetric positive semi-definite G, lambda_max(G)^(2^k) <=
// ||G^(2^k)||_F. Squaring G k times (FP64, renormalised each time) therefore
// bounds sigma_max from above, approaching it as k grows; k = 5 is within a
// fraction of a percent for the weight matrices here. A relative margin of
// 1e-6 covers the FP64 rounding of the products.
#include "launch.h"

#include <cmath>
#include <vector>

namespace vbmc {
namespace {

// C = A * B^T for row-major A [M x K] and B [N x K], FP64 (small set-up GEMMs).
__global__ void k_gemm_abt64(const double* A, const double* B, double* C, int M, int N, int K) {
    __shared__ double As[16][17], Bs[16][17];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    double acc = 0.0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        As[ty][tx] = (row < M && k0 + tx < K) ? A[(size_t)row * K + k0 + tx] : 0.0;
        Bs[ty][tx] = (blockIdx.x * 16 + ty < N && k0 + tx < K)
                         ? B[(size_t)(blockIdx.x * 16 + ty) * K + k0 + tx]
                         : 0.0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) acc += As[ty][k] * Bs[tx][k];
        __syncthreads();
    }
    if (row < M && col < N) C[(size_t)row * N + col] = acc;
}

// Rigorous upper bound of the spectral norm of A (m x n, host, row-major):
// sigma^2 = lambda_max(G) <= ||G^(2^k)||_F^(1/2^k) for the Gram matrix G.
double spectral_bound_impl(const std::vector<double>& A, int m, int n) {
    const bool rows = m <= n;  // G = A A^T (m x m) or A^T A (n x n)
    const int g = rows ? m : n;
    std::vector<double> At;
    const std::vector<double>* src = &A;
    int K = n;
    if (!rows) {
        At.resize((size_t)n * m);
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) At[(size_t)j * m + i] = A[(size_t)i * n + j];
        src = &At;
        K = m;
    }
    double *dA = nullptr, *dG = nullptr, *dH = nullptr;
    cudaMalloc(&dA, sizeof(double) * src->size());
    cudaMalloc(&dG, sizeof(double) * (size_t)g * g);
    cudaMalloc(&dH, sizeof(double) * (size_t)g * g);
    cudaMemcpy(dA, src->data(), sizeof(double) * src->size(), cudaMemcpyHostToDevice);
    dim3 blk(16, 16), grd((g + 15) / 16, (g + 15) / 16);
    k_gemm_abt64<<<grd, blk>>>(dA, dA, dG, g, g, K);
    std::vector<double> h((size_t)g * g);
    double logscale = 0.0;
    const int squarings = 5;
    for (int it = 0; it <= squarings; ++it) {
        cudaMemcpy(h.data(), dG, sizeof(double) * h.size(), cudaMemcpyDeviceToHost);
        double f = 0.0;
        for (double x : h) f += x * x;
        f = std::sqrt(f);
        if (!(f > 0.0)) {
            cudaFree(dA);
            cudaFree(dG);
            cudaFree(dH);
            return 0.0;
        }
        // G_it = exp(logscale) * (current matrix); track the scale, normalise
        logscale = (it == 0 ? 0.0 : 2.0 * logscale) + std::log(f);
        for (double& x : h) x /= f;
        if (it == squarings) break;
        cudaMemcpy(dG, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice);
        k_gemm_abt64<<<grd, blk>>>(dG, dG, dH, g, g, g);  // G symmetric: G G^T = G^2
        std::swap(dG, dH);
    }
    cudaFree(dA);
    cudaFree(dG);
    cudaFree(dH);
    // ||G^(2^k)||_F = exp(logscale); lambda_max <= exp(logscale / 2^k)
    const double lam = std::exp(logscale / (double)(1 << squarings));
    return std::sqrt(lam) * (1.0 + 1e-6);
}

}  // namespace

double spectral_bound(const std::vector<double>& A, int m, int n) { return spectral_bound_impl(A, m, n); }

}  // namespace vbmc
