#define XL_REAL double
#include "xl_rs_inst.cuh"
