#define XL_REAL double
#include "xl_asczt_inst.cuh"
