// screen_simt.cu -- shape dispatch of the FP32 SIMT screen (kernel in screen_simt.cuh).
#include "screen_simt.cuh"

namespace vbmc {

#define VB_SIMT_DECL(i)                                                                            \
    void launch_simt_v##i(const NetView&, const QueryView*, int, const unsigned long long*,      \
                          unsigned long long, const QEntry*, const unsigned long long*,          \
                          unsigned long long, Queue, int, int, cudaStream_t);
VB_SIMT_DECL(1)
VB_SIMT_DECL(2)
VB_SIMT_DECL(3)
VB_SIMT_DECL(4)

int simt_variant(const NetView& net) {
    if (net.hmax <= 32) return 1;
    if (net.hmax <= 256) return 2;
    if (net.hmax <= 512) return 3;
    if (net.hmax <= 1024) return 4;
    return 0;
}

int simt_tile_points(const NetView& net) {
    switch (simt_variant(net)) {
        case 1: return simt::SimtSmem<16, 1>::MT;
        case 2: return simt::SimtSmem<16, 8>::MT;
        case 3: return simt::SimtSmem<8, 16>::MT;
        case 4: return simt::SimtSmem<4, 32>::MT;
    }
    return 0;
}

void launch_screen_simt(const NetView& net, const QueryView* d_qs, int nq,
                        const unsigned long long* tp, unsigned long long n_tiles,
                        const QEntry* gather, const unsigned long long* gc,
                        unsigned long long gcap, Queue out, int level, int n_sm,
                        cudaStream_t st) {
    switch (simt_variant(net)) {
        case 1: launch_simt_v1(net, d_qs, nq, tp, n_tiles, gather, gc, gcap, out, level, n_sm, st); break;
        case 2: launch_simt_v2(net, d_qs, nq, tp, n_tiles, gather, gc, gcap, out, level, n_sm, st); break;
        case 3: launch_simt_v3(net, d_qs, nq, tp, n_tiles, gather, gc, gcap, out, level, n_sm, st); break;
        case 4: launch_simt_v4(net, d_qs, nq, tp, n_tiles, gather, gc, gcap, out, level, n_sm, st); break;
        default: break;
    }
}

}  // namespace vbmc
