// DhopEO/DhopOE kernels, P16 storage.
#define DWF_PREC P16
#include "dhop_inst.cuh"
