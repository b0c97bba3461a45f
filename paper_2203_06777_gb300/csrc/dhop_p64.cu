// DhopEO/DhopOE kernels, P64 storage.
#define DWF_PREC P64
#include "dhop_inst.cuh"
