// DhopEO/DhopOE kernels, P32 storage.
#define DWF_PREC P32
#include "dhop_inst.cuh"
