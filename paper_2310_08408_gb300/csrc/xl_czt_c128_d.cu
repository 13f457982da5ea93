// CZT window-pass kernels of one group of transform lengths (see xl_czt_inst.cuh).
#define XL_REAL double
#define XL_CZT_LENGTHS(X) X(8192)
#include <algorithm>
#include "xl_czt_inst.cuh"
