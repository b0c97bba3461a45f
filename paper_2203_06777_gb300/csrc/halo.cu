// Face assembly for a lattice split into blocks along t (the paper's Section 3: the face-assembly
// kernels of its multi-GPU runs, overlapped with the interior of the hopping term). A block's hop
// out of its last t-plane needs psi(x + t) from the next block's first plane, and out of its
// first plane U_t(x - t)^+ psi(x - t) from the previous block's last plane. Only the spin
// projection of those spinors enters the hop, so a block sends its first plane projected with the
// forward-hop projector (to the previous block) and its last plane with the backward-hop projector
// (to the next one): per site and slice pair 12 complex FP32 values, the exact FP32 values the
// hopping kernel would form itself, so the receiving block's result equals the unsplit lattice's
// bit for bit. A face that crosses the global lattice edge carries the boundary phase, applied
// here by the sender. Face layout: [face site f][j 0..5][pair q] of float4, vector j holding reals
// 2j and 2j + 1 of the half spinor, each for both slices of the pair (2q, 2q + 1); f = cb index
// of the site within its t-plane.
#include "dhop_kernel.cuh"

namespace gdwf {

template <int P, bool DAG>
__global__ void __launch_bounds__(128) k_face_project(const char* in, Geom g, int plane, float ph_first, float ph_last,
                                                      float4* send_first, float4* send_last) {
  using T = typename Store<P>::T;
  constexpr int SF = DAG ? +1 : -1;  // forward-hop projector (1 + SF gamma_t), as in the hop kernel
  constexpr int SB = -SF;
  const int Lsh = ls_half(g.Ls);
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (tid >= 2L * plane * Lsh) return;
  const int q = (int)(tid % Lsh);
  const long rest = tid / Lsh;
  const bool last = rest >= plane;
  const int f = (int)(last ? rest - plane : rest);
  const int site = last ? g.N4h - plane + f : f;
  const char* blk = in + site_offset(site, Lsh, (size_t)Lsh * 2 * 24 * sizeof(T));
  float2 h[12];
  if constexpr (P == P32) {
    float2 psi[24];
    load_pair<P, 0>(blk, q, Lsh, psi);
    if (last)
      project2<SB>(3, psi, h);
    else
      project2<SF>(3, psi, h);
  } else {
    uint32_t w[24];
    load_words<P, 0>(blk, q, Lsh, w);
    if (last)
      project2w<P, SB>(3, w, h);
    else
      project2w<P, SF>(3, w, h);
  }
  const float ph = last ? ph_last : ph_first;  // +1 or -1: exact
  float4* dst = (last ? send_last : send_first) + (size_t)f * 6 * Lsh + q;
#pragma unroll
  for (int j = 0; j < 6; ++j)
    dst[(size_t)j * Lsh] = make_float4(ph * h[2 * j].x, ph * h[2 * j].y, ph * h[2 * j + 1].x, ph * h[2 * j + 1].y);
}

cudaError_t launch_face_project(int prec, bool dag, const Geom& g, int plane, const void* in, float ph_first,
                                float ph_last, void* send_first, void* send_last, cudaStream_t st) {
  const long n = 2L * plane * ls_half(g.Ls);
  const int blocks = (int)((n + 127) / 128);
  const char* i = static_cast<const char*>(in);
  float4* a = static_cast<float4*>(send_first);
  float4* b = static_cast<float4*>(send_last);
#define FP(P_)                                                                                     \
  if (dag)                                                                                         \
    k_face_project<P_, true><<<blocks, 128, 0, st>>>(i, g, plane, ph_first, ph_last, a, b);        \
  else                                                                                             \
    k_face_project<P_, false><<<blocks, 128, 0, st>>>(i, g, plane, ph_first, ph_last, a, b);
  switch (prec) {
    case P32: FP(P32) break;
    case P16: FP(P16) break;
    case PB16: FP(PB16) break;
    default: return cudaErrorInvalidValue;
  }
#undef FP
  return cudaGetLastError();
}

}  // namespace gdwf
