// The FP64 hopping term in float-float arithmetic (dhop_ff.cu): the same DhopArgs and launch
// shape as the FP64 kernel of dhop_kernel.cuh (one thread per (site, slice)), its own
// shared-memory size.
#pragma once

#include "dhop_kernel.cuh"

namespace gdwf {

size_t dhop_ff_smem_bytes(int sites_per_cta, int Ls, bool post);
cudaError_t launch_dhop_ff(const DhopArgs& a, bool dag, bool c12, int threads, int blocks, size_t smem,
                           cudaStream_t stream);

}  // namespace gdwf
