// noalloc.cu -- an FP64 range check that allocates no device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside another
// runtime's memory pool, under a strict memory budget, or in a process whose
// allocator must not be re-entered. For them this entry point keeps every
// piece of per-query scratch (the query view, the validated pixel list, the
// clipped step table, the FP64 potentials of the unperturbed image and the
// counters) in one file-scope __device__ array of kScratchBytes, and writes
// the results only into buffers the caller passes in.
//
// The array lives on every GPU that loads this library until the process
// exits. Host code must not hand its name to a kernel: on the host the name
// is only a stand-in symbol. The first call on each device looks up the
// array's device address with cudaGetSymbolAddress (with that device
// current) and caches it; make that first call before any stream capture.
// All calls share the array, so calls whose work overlaps on the GPU race;
// each call resets everything it relies on before use.
#include "../../include/vbmc.h"
#include "dev.cuh"
#include "launch.h"

#include <cfloat>
#include <cstring>
#include <mutex>
#include <string>

namespace vbmc {
namespace {

constexpr size_t kScratchBytes = 128 * 1024;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Scratch layout (byte offsets, each 256-aligned).
struct Layout {
    size_t qv, cnt, pix, dv, ub, hb, eub, end;
};

Layout layout(int total, int sr) {
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    Layout L{};
    size_t o = 0;
    L.qv = o;
    o = al(o + sizeof(QueryView));
    L.cnt = o;
    o = al(o + sizeof(Counters));
    L.pix = o;
    o = al(o + sizeof(int) * kMaxS);
    L.dv = o;
    o = al(o + sizeof(int) * (size_t)sr);
    L.ub = o;
    o = al(o + sizeof(double) * (size_t)total);
    L.hb = o;
    o = al(o + sizeof(double) * (size_t)total);
    L.eub = o;
    o = al(o + sizeof(double) * (size_t)total);
    L.end = o;
    return L;
}

// Class D of the unperturbed image and its margin (lowest index on ties).
__global__ void k_na_class(NetView net, QueryView* qs) {
    QueryView& Q = qs[0];
    const double* y = Q.ub + net.noff[net.L];
    const int HL = net.dims[net.L];
    int D = 0;
    for (int i = 1; i < HL; ++i)
        if (y[i] > y[D]) D = i;
    double mx = -DBL_MAX;
    for (int i = 0; i < HL; ++i)
        if (i != D && y[i] > mx) mx = y[i];
    Q.cnt->D = D;
    Q.cnt->base_margin = y[D] - mx;
}

// Write the query view into the scratch array. The view travels as a kernel
// argument (by value), so no host buffer has to outlive the call.
__global__ void k_na_set(const QueryView q, QueryView* d_q) { *d_q = q; }

// Copy the counters the caller asked for into its buffer.
__global__ void k_na_out(const QueryView* qs, unsigned long long* out) {
    const Counters* c = qs[0].cnt;
    out[0] = c->n_adv;
    out[1] = c->first;
    out[2] = c->n_ties;
    out[3] = (unsigned long long)(unsigned)c->D | ((unsigned long long)c->err << 32);
}

unsigned char* scratch_address() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) return nullptr;
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    return g_addr[dev];
}

}  // namespace

// Device view of a net handle and the thread's error message (api.cu).
const NetView* net_view(const vbmc_net* net);
vbmc_status set_error(vbmc_status st, const char* msg);

}  // namespace vbmc

using namespace vbmc;

extern "C" vbmc_status vbmc_verify_range_fp64_noalloc(const vbmc_net* net, const uint8_t* d_image,
                                                      int32_t s, const int32_t* d_pixels, int32_t k,
                                                      uint64_t lo, uint64_t hi,
                                                      const vbmc_noalloc_out* out, void* stream) {
    if (!net || !d_image || (!d_pixels && s > 0) || !out || !out->counters)
        return set_error(VBMC_ERR_ARG, "null argument");
    if (s < 0 || s > kMaxS || k < 0 || k > VBMC_MAX_K) return set_error(VBMC_ERR_ARG, "s or k out of range");
    const NetView& v = *net_view(net);
    const int R = 2 * k + 1;
    unsigned long long n = 1;
    for (int p = 0; p < s; ++p) {
        if (n > (1ull << 62) / (unsigned long long)R) return set_error(VBMC_ERR_ARG, "R^s too large");
        n *= (unsigned long long)R;
    }
    if (hi == 0) hi = n;
    if (hi > n || lo > hi) return set_error(VBMC_ERR_ARG, "range [lo, hi) outside [0, R^s)");
    const Layout Ly = layout(v.total, s * R);
    if (Ly.end > kScratchBytes || v.total > VBMC_NOALLOC_MAX_NEURONS || s * R > VBMC_NOALLOC_MAX_SR)
        return set_error(VBMC_ERR_UNSUPPORTED,
                         "query too large for the fixed scratch (VBMC_NOALLOC_MAX_NEURONS non-input "
                         "neurons, s*(2k+1) <= VBMC_NOALLOC_MAX_SR)");
    if (out->bitmap && hi > out->bitmap_bits) return set_error(VBMC_ERR_ARG, "bitmap too small");
    if (out->ties_cap && !out->ties) return set_error(VBMC_ERR_ARG, "ties_cap without ties buffer");
    unsigned char* base = scratch_address();
    if (!base) return set_error(VBMC_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    cudaStream_t st = (cudaStream_t)stream;

    QueryView q{};
    q.s = s;
    q.k = k;
    q.R = R;
    q.qid = 0;
    q.n_points = n;
    q.lo = lo;
    q.hi = hi;
    q.image = d_image;
    q.pix_in = d_pixels;
    q.pix = reinterpret_cast<int*>(base + Ly.pix);
    q.dv = reinterpret_cast<int*>(base + Ly.dv);
    q.ub = reinterpret_cast<double*>(base + Ly.ub);
    q.hb = reinterpret_cast<double*>(base + Ly.hb);
    q.eub = reinterpret_cast<double*>(base + Ly.eub);
    q.cnt = reinterpret_cast<Counters*>(base + Ly.cnt);
    q.bitmap = out->bitmap;
    q.bitmap_bits = out->bitmap ? out->bitmap_bits : 0;
    q.flip = out->flip;
    q.flip_tie = out->flip_tie;
    q.ss = out->ss;
    q.ss_tie = out->ss_tie;
    q.ties = reinterpret_cast<unsigned long long*>(out->ties);
    q.ties_cap = out->ties_cap;
    QueryView* d_q = reinterpret_cast<QueryView*>(base + Ly.qv);
    // coverage needs all four masks; with any missing none is written
    const bool cov = out->flip && out->flip_tie && out->ss && out->ss_tie;
    if (!cov) q.flip = q.flip_tie = q.ss = q.ss_tie = nullptr;
    k_na_set<<<1, 1, 0, st>>>(q, d_q);
    // the caller's result buffers start from zero on every call
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && cov) e = cudaMemsetAsync(out->flip, 0, 4ull * v.flip_words, st);
    if (e == cudaSuccess && cov) e = cudaMemsetAsync(out->flip_tie, 0, 4ull * v.flip_words, st);
    if (e == cudaSuccess && cov) e = cudaMemsetAsync(out->ss, 0, 4ull * v.ss_words, st);
    if (e == cudaSuccess && cov) e = cudaMemsetAsync(out->ss_tie, 0, 4ull * v.ss_words, st);
    if (e == cudaSuccess && out->bitmap && hi > 0)
        e = cudaMemsetAsync(out->bitmap, 0, 4ull * ((hi + 31) / 32), st);
    if (e != cudaSuccess) return set_error(VBMC_ERR_CUDA, cudaGetErrorString(e));
    // k_pro_init resets the counters in the scratch and validates the pixels
    launch_pro_init(v, d_q, 1, st);
    for (int l = 1; l <= v.L; ++l) launch_pro_layer(v, d_q, 1, l, st);
    k_na_class<<<1, 1, 0, st>>>(v, d_q);
    if (hi > lo) {
        int n_sm = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        launch_fp64(v, d_q, 1, nullptr, nullptr, 0, lo, hi, n_sm, st);
    }
    k_na_out<<<1, 1, 0, st>>>(d_q, reinterpret_cast<unsigned long long*>(out->counters));
    const cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) return set_error(VBMC_ERR_CUDA, cudaGetErrorString(le));
    return VBMC_OK;
}
