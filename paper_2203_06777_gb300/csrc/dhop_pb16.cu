// DhopEO/DhopOE kernels, PB16 storage.
#define DWF_PREC PB16
#include "dhop_inst.cuh"
