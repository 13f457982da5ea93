// Launchers of the CZT / VCZT kernels, instantiated once per precision (xl_czt_c64.cu,
// xl_czt_c128.cu).
#pragma once

#include "xl_czt_kernels.cuh"
#include "xl_runtime.h"

namespace xl {

enum { CZT_FWD_X = 0, CZT_FWD_Y = 1, CZT_ADJ_Y = 2, CZT_ADJ_X = 3 };

// One pass of length L (64..8192) over nbatch elements.
template <typename T>
xl_status czt_pass(int which, bool vec, int L, const void* src, void* dst, const CztDims& d,
                   const AxisRun<cplx<T>>& axis, int nbatch, cudaStream_t s);
// Scalar complex64 forward (both passes) through the row-major intermediate Tr[ny][mx] (same size
// as the transposed one): the y pass gathers its columns with bulk tensor copies. mx even,
// lengths 256..8192.
template <typename T>
xl_status czt_fwd_rm(int Lx, int Ly, const void* src, void* Tr, void* dst, const CztDims& d,
                     const AxisRun<cplx<T>>& ax, const AxisRun<cplx<T>>& ay, int nbatch, cudaStream_t s);
// Fills the chirp tables (both axes) and transforms the b rows in place.
template <typename T>
xl_status czt_tables(void* tab, const CztTabArgs& a, cudaStream_t s);
// The same for the angular-spectrum reading (window sums of a centred spectrum; no distance).
template <typename T>
xl_status asczt_tables(void* tab, const CztTabArgs& a, cudaStream_t s);

}  // namespace xl
