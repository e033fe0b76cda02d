// Learned subgrid closure: network shape and parameter layout shared by the training and the
// inference kernels.
#pragma once
#include <cstddef>

namespace erfk {

constexpr int CL_NIN = 12, CL_NH = 64, CL_NOUT = 9;
constexpr int CL_NPARAM = CL_NH * CL_NIN + CL_NH + 2 * (CL_NH * CL_NH + CL_NH) + CL_NOUT * CL_NH + CL_NOUT;  // 9737
// closure blob (host): magic, version, then FP32 in_mean[12] in_std[12] out_mean[9] out_std[9] params[9737]
constexpr unsigned CL_MAGIC = 0x4D465245u;   // "ERFM"
constexpr int CL_BLOB_FLOATS = 2 * CL_NIN + 2 * CL_NOUT + CL_NPARAM;

size_t train_scratch_floats(int batch);

}  // namespace erfk
