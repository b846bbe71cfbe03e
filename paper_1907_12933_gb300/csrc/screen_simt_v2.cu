// screen_simt_v2.cu -- FP32 screen instantiation for widths <= 256 (128 points per tile).
#include "screen_simt.cuh"

namespace vbmc {
void launch_simt_v2(const NetView& net, const QueryView* d_qs, int nq, const unsigned long long* tp,
                     unsigned long long n_tiles, const QEntry* gather, const unsigned long long* gc,
                     unsigned long long gcap, Queue out, int level, int n_sm, cudaStream_t st,
                     unsigned long long* claim) {
    simt::launch_variant<16, 8>(net, d_qs, nq, tp, n_tiles, gather, gc, gcap, out, level, n_sm, st, claim);
}
}  // namespace vbmc
