// CZT window-pass kernels of one group of transform lengths (see xl_czt_inst.cuh).
#define XL_REAL float
#define XL_CZT_LENGTHS(X) X(64) X(128) X(256) X(512)
#include <algorithm>
#include "xl_czt_inst.cuh"
