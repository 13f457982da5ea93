#define XL_REAL float
#include "xl_asczt_inst.cuh"
