#define XL_REAL float
#include "xl_rs_inst.cuh"
