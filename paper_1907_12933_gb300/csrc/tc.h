// tc.h -- tensor-core (tcgen05) screen of layers 2..L (internal).
#pragma once
#include "../../include/vbmc.h"
#include "dev.cuh"

#include <vector>

namespace vbmc {

struct TcNet {
    void* d_wq[kMaxL + 1] = {};  // quantised weights per layer and precision (see tc.cu)
    void* d_wlo[kMaxL + 1] = {};
    float* d_consts = nullptr;
    std::vector<void*> owned;
};

bool tc_supported(const NetView& v, int precision);
vbmc_status tc_build(TcNet& tc, const NetView& v, const std::vector<std::vector<float>>& W,
                     const std::vector<std::vector<float>>& b);
void tc_free(TcNet& tc);
vbmc_status tc_launch_screen(TcNet& tc, const NetView& v, const QueryView* d_q, uint64_t lo,
                             uint64_t hi, int precision, Queue out, int n_sm, cudaStream_t st);
vbmc_status tc_launch_gather(TcNet& tc, const NetView& v, const QueryView* d_q, const QEntry* in,
                             const unsigned long long* in_count, unsigned long long cap,
                             int precision, Queue out, int n_sm, cudaStream_t st);

}  // namespace vbmc
