#define XL_REAL double
#include <algorithm>
#include "xl_czt_inst.cuh"
