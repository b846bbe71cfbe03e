// tc.cu -- tensor-core screen (tcgen05). Placeholder until the kernel lands.
#include "tc.h"

namespace vbmc {

bool tc_supported(const NetView&, int) { return false; }
vbmc_status tc_build(TcNet&, const NetView&, const std::vector<std::vector<float>>&,
                     const std::vector<std::vector<float>>&) {
    return VBMC_ERR_UNSUPPORTED;
}
void tc_free(TcNet& tc) {
    for (void* p : tc.owned) cudaFree(p);
    tc.owned.clear();
}
vbmc_status tc_launch_screen(TcNet&, const NetView&, const QueryView*, uint64_t, uint64_t, int, Queue,
                             int, cudaStream_t) {
    return VBMC_ERR_UNSUPPORTED;
}
vbmc_status tc_launch_gather(TcNet&, const NetView&, const QueryView*, const QEntry*,
                             const unsigned long long*, unsigned long long, int, Queue, int,
                             cudaStream_t) {
    return VBMC_ERR_UNSUPPORTED;
}

}  // namespace vbmc
