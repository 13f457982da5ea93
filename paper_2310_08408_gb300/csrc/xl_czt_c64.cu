#define XL_REAL float
#include <algorithm>
#include "xl_czt_inst.cuh"
