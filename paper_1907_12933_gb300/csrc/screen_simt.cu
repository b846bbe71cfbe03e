// screen_simt.cu -- shape dispatch of the FP32 SIMT screen (kernel in screen_simt.cuh).
#include "screen_simt.cuh"

namespace vbmc {

#define VB_SIMT_DECL(i)                                                                            \
    void launch_simt_v##i(const NetView&, const QueryView*, int, const unsigned long long*,      \
                          unsigned long long, const QEntry*, const unsigned long long*,          \
                          unsigned long long, Queue, int, int, cudaStream_t, unsigned long long*);
VB_SIMT_DECL(1)
VB_SIMT_DECL(2)
VB_SIMT_DECL(3)
VB_SIMT_DECL(4)
VB_SIMT_DECL(5)
VB_SIMT_DECL(6)

// Widest layer each variant holds: 32 * NQ neurons (NQ accumulators per lane).
// Variants 5 and 6 hold the widths of 3 and 2 with half the points per tile
// (fewer registers and less shared memory: more CTAs per SM).
int simt_variant_width(int var) {
    switch (var) {
        case 1: return 32;
        case 2: return 256;
        case 3: return 512;
        case 4: return 1024;
        case 5: return 512;
        case 6: return 256;
    }
    return 0;
}

// The narrowest variant that holds the net's widest layer.
int simt_variant_default(const NetView& net) {
    for (int var = 1; var <= 4; ++var)
        if (net.hmax <= simt_variant_width(var)) return var;
    return 0;
}

// Variant of the range passes (tuned, else the narrowest that fits).
int simt_variant(const NetView& net) {
    const int t = net.simt_var_range;
    return (t >= 1 && t <= kSimtVariants && net.hmax <= simt_variant_width(t)) ? t : simt_variant_default(net);
}

int simt_variant_points(int var) {
    switch (var) {
        case 1: return simt::SimtSmem<16, 1>::MT;
        case 2: return simt::SimtSmem<16, 8>::MT;
        case 3: return simt::SimtSmem<8, 16>::MT;
        case 4: return simt::SimtSmem<4, 32>::MT;
        case 5: return simt::SimtSmem<4, 16>::MT;
        case 6: return simt::SimtSmem<8, 8>::MT;
    }
    return 0;
}

int simt_tile_points(const NetView& net) { return simt_variant_points(simt_variant(net)); }

size_t simt_variant_smem(int var) {
    switch (var) {
        case 1: return sizeof(simt::SimtSmem<16, 1>);
        case 2: return sizeof(simt::SimtSmem<16, 8>);
        case 3: return sizeof(simt::SimtSmem<8, 16>);
        case 4: return sizeof(simt::SimtSmem<4, 32>);
        case 5: return sizeof(simt::SimtSmem<4, 16>);
        case 6: return sizeof(simt::SimtSmem<8, 8>);
    }
    return 0;
}

void launch_screen_simt(const NetView& net, const QueryView* d_qs, int nq,
                        const unsigned long long* tp, unsigned long long n_tiles,
                        const QEntry* gather, const unsigned long long* gc,
                        unsigned long long gcap, Queue out, int level, int n_sm,
                        cudaStream_t st, unsigned long long* claim) {
    if (nq == 1 && small_supported(net)) {  // one thread per point
        launch_small(net, d_qs, tp, n_tiles, gather, gc, gcap, out, level, n_sm, st);
        return;
    }
    if (claim && !gather && cudaMemsetAsync(claim, 0, sizeof(unsigned long long), st) != cudaSuccess) return;
    int var = simt_variant(net);
    if (gather) {
        const int t = net.simt_var_gather;
        var = (t >= 1 && t <= kSimtVariants && net.hmax <= simt_variant_width(t)) ? t : simt_variant_default(net);
    }
    switch (var) {
        case 1: launch_simt_v1(net, d_qs, nq, tp, n_tiles, gather, gc, gcap, out, level, n_sm, st, claim); break;
        case 2: launch_simt_v2(net, d_qs, nq, tp, n_tiles, gather, gc, gcap, out, level, n_sm, st, claim); break;
        case 3: launch_simt_v3(net, d_qs, nq, tp, n_tiles, gather, gc, gcap, out, level, n_sm, st, claim); break;
        case 4: launch_simt_v4(net, d_qs, nq, tp, n_tiles, gather, gc, gcap, out, level, n_sm, st, claim); break;
        case 5: launch_simt_v5(net, d_qs, nq, tp, n_tiles, gather, gc, gcap, out, level, n_sm, st, claim); break;
        case 6: launch_simt_v6(net, d_qs, nq, tp, n_tiles, gather, gc, gcap, out, level, n_sm, st, claim); break;
        default: break;
    }
}

}  // namespace vbmc
