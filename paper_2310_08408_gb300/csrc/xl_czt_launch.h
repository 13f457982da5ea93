// Launchers of the CZT / VCZT kernels, instantiated once per precision (xl_czt_c64.cu,
// xl_czt_c128.cu).
#pragma once

#include "xl_czt_kernels.cuh"
#include "xl_runtime.h"

namespace xl {

enum { CZT_FWD_X = 0, CZT_FWD_Y = 1, CZT_ADJ_Y = 2, CZT_ADJ_X = 3 };

// Segment plan of one axis (N grid samples -> M window samples): transform length L, S segments
// of `seg` samples. Chosen to minimise the (S + 1) L log2 L transform work among the plans whose
// shared memory fits (the same plan for every call of the same sizes, precision and mode).
struct CztAxisPlan {
  int L, S, seg;
};
CztAxisPlan czt_axis_plan(int N, int M, int csize, bool vec, bool dz);

// Extra arguments of the distance-gradient kernels (the `dz` forms of the passes).
template <typename C> struct CztDzArgs {
  CztSaved<C> sv;     // what the forward saves (read by the adjoint passes)
  double* dzp;        // adjoint passes: partial sums [b][block][6 or 2]
  const C* u_in;      // adjoint x pass: the forward input
  bool on;            // the passes run their DZ form
};

// One pass of length L (64..8192) over nbatch elements.
template <typename T>
xl_status czt_pass(int which, bool vec, int L, const void* src, void* dst, const CztDims& d,
                   const AxisRun<cplx<T>>& axis, int nbatch, cudaStream_t s,
                   const CztDzArgs<cplx<T>>* dz = nullptr, int* blocks = nullptr);
// Scalar complex64 forward (both passes) through the row-major intermediate Tr[ny][mx] (same size
// as the transposed one): the y pass gathers its columns with bulk tensor copies. mx even,
// lengths 256..8192, one segment per axis.
template <typename T>
xl_status czt_fwd_rm(int Lx, int Ly, const void* src, void* Tr, void* dst, const CztDims& d,
                     const AxisRun<cplx<T>>& ax, const AxisRun<cplx<T>>& ay, int nbatch, cudaStream_t s);
// Fills the chirp tables (both axes) and transforms the b rows in place.
template <typename T>
xl_status czt_tables(void* tab, const CztTabArgs& a, cudaStream_t s);
// The same for the angular-spectrum reading (window sums of a centred spectrum; no distance).
template <typename T>
xl_status asczt_tables(void* tab, const CztTabArgs& a, cudaStream_t s);
// Distance gradients of a launch's elements from the adjoint passes' partial sums.
xl_status czt_dz_finalize(const double* py, int nby, const double* px, int nbx, const double* zdev,
                          const CztDims& d, double k, bool phase_invariant, double* g_z, int nb,
                          cudaStream_t s);

}  // namespace xl
