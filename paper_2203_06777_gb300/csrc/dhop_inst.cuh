// Instantiates launch_dhop<DWF_PREC>: one translation unit per storage precision so that the
// kernel variants of the four precisions compile in parallel.
#include "dhop_kernel.cuh"

namespace gdwf {

template <int ST, bool DAG, bool C12>
static cudaError_t launch_one(const DhopArgs& a, int threads, int blocks, size_t smem, cudaStream_t stream) {
  auto kern = dhop_kernel<DWF_PREC, ST, DAG, C12>;
  if (smem > 48 * 1024) {
    static size_t configured = 0;  // per instantiation
    if (smem > configured) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      configured = smem;
    }
  }
  kern<<<blocks, threads, smem, stream>>>(a);
  return cudaGetLastError();
}

template <>
cudaError_t launch_dhop<DWF_PREC>(const DhopArgs& a, int st, bool dag, bool c12, int threads, int blocks, size_t smem,
                                  cudaStream_t stream) {
#define DWF_DISPATCH(ST_)                                                         \
  if (dag) return c12 ? launch_one<ST_, true, true>(a, threads, blocks, smem, stream) \
                      : launch_one<ST_, true, false>(a, threads, blocks, smem, stream); \
  return c12 ? launch_one<ST_, false, true>(a, threads, blocks, smem, stream)         \
             : launch_one<ST_, false, false>(a, threads, blocks, smem, stream);
  if (st == 2) {
    DWF_DISPATCH(2)
  }
  DWF_DISPATCH(1)
#undef DWF_DISPATCH
}

}  // namespace gdwf
