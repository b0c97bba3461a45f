// Instantiates launch_dhop<DWF_PREC>: one translation unit per storage precision so that the
// kernel variants of the four precisions compile in parallel.
#include "dhop_pipe.cuh"

namespace gdwf {

template <bool DAG, bool C12, int LSC>
static cudaError_t launch_one(const DhopArgs& a, int threads, int blocks, size_t smem, cudaStream_t stream) {
  auto kern = dhop_kernel<DWF_PREC, DAG, C12, LSC>;
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

// Persistent pipelined kernel: as many CTAs as fit on the device at once (at most one per tile).
template <bool DAG, bool C12, int LSC>
static cudaError_t launch_pipe(const DhopArgs& a, int threads, size_t smem, cudaStream_t stream) {
  auto kern = dhop_pipe_kernel<DWF_PREC, DAG, C12, LSC>;
  static size_t configured = 0;  // per instantiation
  static size_t occ_smem = 0;
  static int occ = 0, sms = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  if (occ_smem != smem || occ == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    occ_smem = smem;
  }
  const PipePlan pl = pipe_plan(a.g, a.pipe_rows, a.pipe_slots, (int)sizeof(typename Store<DWF_PREC>::T),
                                link_bytes(sizeof(typename Store<DWF_PREC>::T), C12), a.pre != PRE_NONE,
                                a.post != POST_NONE);
  const int blocks = pl.tiles < occ * sms ? pl.tiles : occ * sms;
  kern<<<blocks, threads, smem, stream>>>(a);
  return cudaGetLastError();
}

template <int LSC>
static cudaError_t launch_ls(const DhopArgs& a, bool dag, bool c12, int threads, int blocks, size_t smem,
                             cudaStream_t stream) {
  if constexpr (LSC > 0 && DWF_PREC != P64) {
    if (a.pipe_rows > 0) {
      if (dag) return c12 ? launch_pipe<true, true, LSC>(a, threads, smem, stream)
                          : launch_pipe<true, false, LSC>(a, threads, smem, stream);
      return c12 ? launch_pipe<false, true, LSC>(a, threads, smem, stream)
                 : launch_pipe<false, false, LSC>(a, threads, smem, stream);
    }
    if (a.seg > 0) {
      if (dag) return c12 ? launch_tma<true, true, LSC>(a, threads, blocks, smem, stream)
                          : launch_tma<true, false, LSC>(a, threads, blocks, smem, stream);
      return c12 ? launch_tma<false, true, LSC>(a, threads, blocks, smem, stream)
                 : launch_tma<false, false, LSC>(a, threads, blocks, smem, stream);
    }
  }
  if (dag) return c12 ? launch_one<true, true, LSC>(a, threads, blocks, smem, stream)
                      : launch_one<true, false, LSC>(a, threads, blocks, smem, stream);
  return c12 ? launch_one<false, true, LSC>(a, threads, blocks, smem, stream)
             : launch_one<false, false, LSC>(a, threads, blocks, smem, stream);
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
