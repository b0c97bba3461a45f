// Instantiates launch_dhop<DWF_PREC>: one translation unit per storage precision so that the
// kernel variants of the four precisions compile in parallel.
#include "dhop_tma.cuh"

namespace gdwf {

template <bool DAG, bool C12, int LSC, bool EPI>
static cudaError_t launch_one(const DhopArgs& a, int threads, int blocks, size_t smem, cudaStream_t stream) {
  auto kern = dhop_kernel<DWF_PREC, DAG, C12, LSC, EPI>;
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

template <bool DAG, bool C12, int LSC>
static cudaError_t launch_tma(const DhopArgs& a, int threads, int blocks, size_t smem, cudaStream_t stream) {
  auto kern = dhop_tma_kernel<DWF_PREC, DAG, C12, LSC>;
  static size_t configured = 0;  // per instantiation
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  kern<<<blocks, threads, smem, stream>>>(a);
  return cudaGetLastError();
}

template <int LSC>
static cudaError_t launch_ls(const DhopArgs& a, bool dag, bool c12, int threads, int blocks, size_t smem,
                             cudaStream_t stream) {
  if constexpr (LSC > 0 && DWF_PREC != P64) {
    if (a.seg > 0) {
      if (dag) return c12 ? launch_tma<true, true, LSC>(a, threads, blocks, smem, stream)
                          : launch_tma<true, false, LSC>(a, threads, blocks, smem, stream);
      return c12 ? launch_tma<false, true, LSC>(a, threads, blocks, smem, stream)
                 : launch_tma<false, false, LSC>(a, threads, blocks, smem, stream);
    }
  }
  // A launch without pre- or post-operation runs the instantiation compiled without the epilogue
  // code (fewer live registers); FP64 always runs the general one.
  const bool epi = DWF_PREC == P64 || a.pre != PRE_NONE || a.post != POST_NONE;
  if (epi) {
    if (dag) return c12 ? launch_one<true, true, LSC, true>(a, threads, blocks, smem, stream)
                        : launch_one<true, false, LSC, true>(a, threads, blocks, smem, stream);
    return c12 ? launch_one<false, true, LSC, true>(a, threads, blocks, smem, stream)
               : launch_one<false, false, LSC, true>(a, threads, blocks, smem, stream);
  }
  if constexpr (DWF_PREC != P64) {
    if (dag) return c12 ? launch_one<true, true, LSC, false>(a, threads, blocks, smem, stream)
                        : launch_one<true, false, LSC, false>(a, threads, blocks, smem, stream);
    return c12 ? launch_one<false, true, LSC, false>(a, threads, blocks, smem, stream)
               : launch_one<false, false, LSC, false>(a, threads, blocks, smem, stream);
  }
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_dhop<DWF_PREC>(const DhopArgs& a, bool dag, bool c12, int threads, int blocks, size_t smem,
                                  cudaStream_t stream) {
  switch (a.g.Ls) {
#define DWF_CASE(L_) \
  case L_:           \
    return launch_ls<L_>(a, dag, c12, threads, blocks, smem, stream);
    DWF_LS_SPECIALISATIONS(DWF_CASE)
#undef DWF_CASE
    default:
      return launch_ls<0>(a, dag, c12, threads, blocks, smem, stream);
  }
}

}  // namespace gdwf
