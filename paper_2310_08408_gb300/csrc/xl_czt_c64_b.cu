// CZT window-pass kernels of one group of transform lengths (see xl_czt_inst.cuh).
#define XL_REAL float
#define XL_CZT_LENGTHS(X) X(1024) X(2048)
#include <algorithm>
#include "xl_czt_inst.cuh"
