// Launchers of the angular-spectrum CZT spectrum passes, instantiated once per precision
// (xl_asczt_c64.cu, xl_asczt_c128.cu).
#pragma once

#include "xl_asczt_kernels.cuh"
#include "xl_runtime.h"

namespace xl {

// forward pass A (stage 0) or B (stage 1): nbatch planes of nrows rows of length L
template <typename T>
xl_status as_fwd_pass(int stage, int L, const void* in, void* out, int nrows, const void* Hc,
                      const AsShift& hs, int nbatch, cudaStream_t s);
// adjoint pass B (stage 1, optionally with the distance partials) or A (stage 0)
template <typename T>
xl_status as_adj_pass(int stage, int L, const void* in, void* out, int nrows, const void* Hc,
                      const void* dHc, const AsShift& hs, const void* TU, double* dz_part,
                      int nbatch, cudaStream_t s);
// blocks per batch element of the adjoint pass B with distance partials
template <typename T> int as_dz_blocks(int L, int nrows);
// transfer tables Hc (and dHc, nullable) of one distance
template <typename T>
xl_status as_transfer(void* Hc, void* dHc, const AsTransferArgs& a, cudaStream_t s);

}  // namespace xl
