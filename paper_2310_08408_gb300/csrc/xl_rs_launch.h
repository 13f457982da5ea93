// Launchers of the RS / VRS kernels, instantiated once per precision (xl_rs_c64.cu,
// xl_rs_c128.cu) so that the two precisions compile in parallel.
#pragma once

#include "xl_rs_kernels.cuh"
#include "xl_runtime.h"

namespace xl {

// pass 1: nplanes input planes [ny][nx] -> T (plane map p -> (p / cin) * cT + p % cin)
template <typename T>
xl_status rs_pass1(const void* in, void* Tb, int nx, int ny, int cin, int cT, int nplanes,
                   cudaStream_t s);
// pass 1 into the row-major intermediate Tr[plane][y][kx] (complex64, rows of 256..8192), read
// by pass 2 of the scalar forward and saved-spectrum adjoint through bulk tensor copies
template <typename T>
xl_status rs_pass1_rm(const void* in, void* Tr, int nx, int ny, int cin, int cT, int nplanes,
                      cudaStream_t s);
// pass 3: T -> nplanes output planes (plane map p -> (p / cout) * cT + p % cout); optionally
// also reduces the pass-2 distance partials (red.part non-null)
template <typename T>
xl_status rs_pass3(const void* Tb, void* out, int nx, int ny, int cout, int cT, int nplanes,
                   cudaStream_t s, DzReduce red = DzReduce{nullptr, 0, nullptr});
// pass 2 over nbatch elements; dz_part gets nbatch * rs_pass2_blocks() partials
// (Tr non-null: the input columns come from the row-major intermediate, modes P2_RS and
// P2_RS_BWD_S of complex64; the results go to Tb)
template <typename T>
xl_status rs_pass2(int mode, void* Tb, const void* Ub, const void* Hq, double* dz_part,
                   const P2Args& a, int nbatch, cudaStream_t s, const void* Tr = nullptr);
template <typename T> int rs_pass2_blocks(int nx, int ny);
// spectrum generation: S scratch ((nx+1) * ny per produced kind), Hq output
template <typename T>
xl_status rs_generate(void* S, void* Hq, const GenArgs& g, int nb, cudaStream_t s);

}  // namespace xl
