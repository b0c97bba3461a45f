// Instantiates launch_dhop<DWF_PREC>: one translation unit per storage precision so that the
// kernel variants of the four precisions compile in parallel.
#include "dhop_kernel.cuh"

namespace gdwf {

template <bool DAG, bool C12, int LSC, int EK>
static cudaError_t launch_one(const DhopArgs& a, int threads, int blocks, size_t smem, cudaStream_t stream) {
  auto kern = dhop_kernel<DWF_PREC, DAG, C12, LSC, EK>;
  if (smem > 48 * 1024) {
    static size_t configured = 0;  // per instantiation
    if (smem > configured) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      configured = smem;
    }
  }
  if constexpr (DWF_PREC == P64) {
    kern<<<blocks, threads, smem, stream>>>(a);
  } else {
    // full CTAs only (the packed kernel has no tail handling); a ragged end gets one more CTA (per
    // half) flush with the end of the lattice, launched after the first so no two writes overlap
    // in time. a.in2 != nullptr: both halves of a full-lattice hop in the same launches.
    // CG epilogues: partial sums [0, halves * full) from the full CTAs (CTA order), then one per
    // half from the end CTAs, which add only the sites the full CTAs did not cover.
    const int nsites = a.region_sites > 0 ? a.region_sites : a.g.N4h;
    const int full = nsites / a.sites_per_cta;
    const int halves = a.in2 ? 2 : 1;
    DhopArgs m = a;
    m.blocks1 = full;
    m.red_base = 0;
    m.own_from = 0;
    if (full > 0) {
      if (a.pdl) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(halves * full);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, kern, m);
        if (e != cudaSuccess) return e;
      } else {
        kern<<<halves * full, threads, smem, stream>>>(m);
      }
    }
    if (a.region_sites == 0 && full * a.sites_per_cta != a.g.N4h) {
      DhopArgs t = a;
      t.site_base = a.g.N4h - a.sites_per_cta;
      t.blocks1 = 1;
      t.red_base = halves * full;
      t.own_from = full * a.sites_per_cta;
      kern<<<halves, threads, smem, stream>>>(t);
    }
  }
  return cudaGetLastError();
}

template <int LSC>
static cudaError_t launch_ls(const DhopArgs& a, bool dag, bool c12, int threads, int blocks, size_t smem,
                             cudaStream_t stream) {
  if constexpr (DWF_PREC == P64) {
    if (dag) return c12 ? launch_one<true, true, LSC, EPI_BOTH>(a, threads, blocks, smem, stream)
                        : launch_one<true, false, LSC, EPI_BOTH>(a, threads, blocks, smem, stream);
    return c12 ? launch_one<false, true, LSC, EPI_BOTH>(a, threads, blocks, smem, stream)
               : launch_one<false, false, LSC, EPI_BOTH>(a, threads, blocks, smem, stream);
  } else {
    // the instantiation with exactly the epilogue parts this launch uses; the CG epilogues exist
    // for the launches that use them only: Mpc's second launch (pre-operation Mooee, no dag) with
    // the norm, Mpc^+'s second launch (Mooee^+, dag) with the update, 18-real links
    if (a.halo_fwd) {  // a face region of a block of a lattice split in t (plain hop)
      if (a.pre != PRE_NONE || a.post != POST_NONE || a.red || a.in2) return cudaErrorInvalidValue;
      if (dag) return c12 ? launch_one<true, true, LSC, EPI_HALO>(a, threads, blocks, smem, stream)
                          : launch_one<true, false, LSC, EPI_HALO>(a, threads, blocks, smem, stream);
      return c12 ? launch_one<false, true, LSC, EPI_HALO>(a, threads, blocks, smem, stream)
                 : launch_one<false, false, LSC, EPI_HALO>(a, threads, blocks, smem, stream);
    }
    if (a.red && !c12 && a.pre != PRE_NONE && a.post == POST_NONE) {
      if (a.r && dag) return launch_one<true, false, LSC, EPI_PRE | EPI_AXPY>(a, threads, blocks, smem, stream);
      if (!a.r && !dag) return launch_one<false, false, LSC, EPI_PRE | EPI_NORM>(a, threads, blocks, smem, stream);
      return cudaErrorInvalidValue;
    }
    if (a.red) return cudaErrorInvalidValue;
    const int ek = (a.pre != PRE_NONE ? EPI_PRE : 0) | (a.post != POST_NONE ? EPI_POST : 0);
#define DWF_EK(K)                                                                             \
  case K:                                                                                     \
    if (dag) return c12 ? launch_one<true, true, LSC, K>(a, threads, blocks, smem, stream)    \
                        : launch_one<true, false, LSC, K>(a, threads, blocks, smem, stream);  \
    return c12 ? launch_one<false, true, LSC, K>(a, threads, blocks, smem, stream)            \
               : launch_one<false, false, LSC, K>(a, threads, blocks, smem, stream);
    switch (ek) {
      DWF_EK(EPI_NONE)
      DWF_EK(EPI_PRE)
      DWF_EK(EPI_POST)
      DWF_EK(EPI_BOTH)
    }
#undef DWF_EK
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
