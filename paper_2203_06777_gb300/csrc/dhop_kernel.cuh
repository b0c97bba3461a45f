// The Wilson hopping stencil on 5D domain-wall fields (DhopEO / DhopOE and their adjoints),
// with optional fused fifth-dimension epilogues.
//
// The paper (Section 3, the Nsight-Compute profile of its main DWF kernel; Conclusion,
// the node-local "Wilson" matrix) identifies this stencil as the memory-bound hot path of the
// domain wall fermion operator. For output sites x of one parity and every slice s:
//
//   Dhop psi(x, s) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu, s) + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu, s)
//
// (dag swaps the projector signs), with the boundary phase bc[mu] on hops that cross the lattice
// edge. gamma matrices are in the chiral basis; the rank-2 projectors (1 +- gamma_mu) are applied
// as "project to a half spinor, multiply by the link, reconstruct", so that each hop costs two
// colour mat-vecs instead of four.
//
// Thread mapping. FP32 and the 16-bit storage formats: one thread per (4D checkerboard site,
// slice pair); every real of the two slices is a float2 and each hop (projection, SU(3)
// product, reconstruction) runs on packed two-wide FP32 instructions, one instruction for two
// slices. FP64: one thread per (site, slice) with scalar arithmetic (the FP64 pipe, not the
// instruction issue, bounds it). All threads of a site load the same link (a broadcast load), so
// every link is read from memory once per site and reused for all Ls slices; a CTA holds whole
// sites, which the fused Mooee^-1 epilogue needs.
//
// Epilogue (all optional, chosen per launch):
//   out = post( alpha * Dhop_in + beta * pre(aux) ),
//   pre  in { none, aux, Mooee aux, Mooee^+ aux },  post in { none, Mooee^-1, (Mooee^+)^-1 },
// with aux a field of the output parity. This fuses the Schur-complement steps
//   t_e = Mooee^-1 D_eo psi_o    and    y_o = Mooee psi_o - D_oe t_e / 4
// into single passes over memory.
#pragma once

#include "dwf_common.cuh"

namespace gdwf {

enum PreOp : int { PRE_NONE = 0, PRE_AUX = 1, PRE_MOOEE = 2, PRE_MOOEE_DAG = 3 };
enum PostOp : int { POST_NONE = 0, POST_INV = 1, POST_INV_DAG = 2 };

struct DhopArgs {
  const void* in;    // input half field (parity 1 - out_parity)
  void* out;         // output half field (parity out_parity)
  const void* aux;   // epilogue input half field (parity out_parity) or null
  const void* Uout;  // links of the output-parity sites (forward hops)
  const void* Uin;   // links of the input-parity sites (backward hops)
  Geom g;
  int out_parity;
  int nsg;            // threads per site (slice pairs, or slices in FP64)
  int sites_per_cta;  // whole sites per CTA
  int pre, post;
  int site_base;      // packed kernels: first site of block 0 (every CTA of a launch is full)
  // Packed kernels, both halves of a full-lattice hop in one launch: CTAs from blocks1 on (or the
  // odd CTAs, with interleave below) apply the other half (output parity 1 - out_parity, fields
  // in2 / out2 / aux2, links swapped). A launch of one half sets blocks1 to its grid size.
  int blocks1;
  const void* in2;
  void* out2;
  const void* aux2;
  // CG epilogues of the packed kernels (EPI_NORM, EPI_AXPY; one half per launch): FP64 partial
  // sums, one per CTA, go to red[red_base + CTA index]; a thread adds nothing (and, for EPI_AXPY,
  // stores nothing) for a site below own_from, which a previous launch already covered.
  int pdl;  // host side: launch the packed kernel as a programmatic dependent of the previous one
  // EPI_HALO (the lattice of this handle is one block of a lattice split in t): the t hops that
  // leave the block read projected half spinors from halo_fwd (beyond the last plane) and
  // halo_bwd (before the first plane), [face site][6][pair] float4 of FP32 values, face site =
  // cb index within the plane; the backward link of the first plane comes from halo_links
  // ([face site], stored link format). plane = checkerboard sites per t-plane.
  const void* halo_fwd;
  const void* halo_bwd;
  const void* halo_links;
  int plane;
  // > 0: the launch covers only region_sites sites from site_base on (a multiple of
  // sites_per_cta; one half), e.g. the interior or one face plane of a block
  int region_sites;
  double* red;
  int red_base;
  int own_from;
  float* r;            // EPI_AXPY: FP32 half field updated in place, r -= (*axpy_coef) * (hopping result)
  const double* axpy_coef;
  // Order in which the CTAs of a packed launch walk the lattice. zblk = 0: lexicographic (CTA b
  // covers cb sites b * sites_per_cta ..). zblk > 0: the (x, y) planes are taken z-fastest within
  // blocks of zblk planes in z, then t, then the next block in z, so that an input plane is
  // reused by the output planes at t - 1, t, t + 1 within about 2 * zblk planes of traffic rather
  // than 2 * Lz (L2 then holds the t-neighbours of lattices whose half field is larger than it).
  // Requires full CTAs tiling each (x, y) plane: ctas_per_plane * sites_per_cta = Lx/2 * Ly.
  int zblk, ctas_per_plane;
  FastDiv div_cpp, div_zblk, div_lt;
  // Full-lattice launches: 1 to alternate the CTAs between the two halves (CTA 2b + h: CTA b of
  // half h) instead of running all CTAs of the first half first.
  int interleave;
  double alpha, beta;
  double d5;       // 5 - M5
  double mass;     // m
  double inv_d5;   // 1 / (5 - M5)
  double inv_den;  // 1 / ((5 - M5) + m (5 - M5)^-(Ls-1))
};

// ---------------------------------------------------------------- spin algebra
// h: half spinor [spin 2][colour 3][re, im]; psi and acc: [spin 4][colour 3][re, im].
// SIG = +1 applies (1 + gamma_mu), SIG = -1 applies (1 - gamma_mu).

template <int SIG, typename R>
__device__ __forceinline__ void project(int mu, const R* psi, R* h) {
#define PR(sp, c) psi[((sp)*3 + (c)) * 2]
#define PI(sp, c) psi[((sp)*3 + (c)) * 2 + 1]
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R h0r, h0i, h1r, h1i;
    if (mu == 0) {  // h0 = psi0 - SIG i psi3, h1 = psi1 - SIG i psi2
      h0r = PR(0, c) + SIG * PI(3, c);
      h0i = PI(0, c) - SIG * PR(3, c);
      h1r = PR(1, c) + SIG * PI(2, c);
      h1i = PI(1, c) - SIG * PR(2, c);
    } else if (mu == 1) {  // h0 = psi0 - SIG psi3, h1 = psi1 + SIG psi2
      h0r = PR(0, c) - SIG * PR(3, c);
      h0i = PI(0, c) - SIG * PI(3, c);
      h1r = PR(1, c) + SIG * PR(2, c);
      h1i = PI(1, c) + SIG * PI(2, c);
    } else if (mu == 2) {  // h0 = psi0 - SIG i psi2, h1 = psi1 + SIG i psi3
      h0r = PR(0, c) + SIG * PI(2, c);
      h0i = PI(0, c) - SIG * PR(2, c);
      h1r = PR(1, c) - SIG * PI(3, c);
      h1i = PI(1, c) + SIG * PR(3, c);
    } else {  // h0 = psi0 + SIG psi2, h1 = psi1 + SIG psi3
      h0r = PR(0, c) + SIG * PR(2, c);
      h0i = PI(0, c) + SIG * PI(2, c);
      h1r = PR(1, c) + SIG * PR(3, c);
      h1i = PI(1, c) + SIG * PI(3, c);
    }
    h[(0 * 3 + c) * 2] = h0r;
    h[(0 * 3 + c) * 2 + 1] = h0i;
    h[(1 * 3 + c) * 2] = h1r;
    h[(1 * 3 + c) * 2 + 1] = h1i;
  }
#undef PR
#undef PI
}

template <typename R>
__device__ __forceinline__ R fma_r(R a, R b, R c);
template <>
__device__ __forceinline__ float fma_r<float>(float a, float b, float c) {
  return fmaf(a, b, c);
}
template <>
__device__ __forceinline__ double fma_r<double>(double a, double b, double c) {
  return fma(a, b, c);
}

// acc += c * reconstruct(uh): upper spins take uh, lower spins the matching multiple of it.
// c carries the boundary phase and any overall scale, so each term is one FMA.
template <int SIG, typename R>
__device__ __forceinline__ void accumulate(int mu, const R* uh, R c, R* acc) {
  const R cs = SIG * c;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const R a0r = uh[(0 * 3 + k) * 2], a0i = uh[(0 * 3 + k) * 2 + 1];
    const R a1r = uh[(1 * 3 + k) * 2], a1i = uh[(1 * 3 + k) * 2 + 1];
    R* s0 = acc + (0 * 3 + k) * 2;
    R* s1 = acc + (1 * 3 + k) * 2;
    R* s2 = acc + (2 * 3 + k) * 2;
    R* s3 = acc + (3 * 3 + k) * 2;
    s0[0] = fma_r(c, a0r, s0[0]);
    s0[1] = fma_r(c, a0i, s0[1]);
    s1[0] = fma_r(c, a1r, s1[0]);
    s1[1] = fma_r(c, a1i, s1[1]);
    if (mu == 0) {  // spin2 += SIG i uh1, spin3 += SIG i uh0
      s2[0] = fma_r(-cs, a1i, s2[0]);
      s2[1] = fma_r(cs, a1r, s2[1]);
      s3[0] = fma_r(-cs, a0i, s3[0]);
      s3[1] = fma_r(cs, a0r, s3[1]);
    } else if (mu == 1) {  // spin2 += SIG uh1, spin3 -= SIG uh0
      s2[0] = fma_r(cs, a1r, s2[0]);
      s2[1] = fma_r(cs, a1i, s2[1]);
      s3[0] = fma_r(-cs, a0r, s3[0]);
      s3[1] = fma_r(-cs, a0i, s3[1]);
    } else if (mu == 2) {  // spin2 += SIG i uh0, spin3 -= SIG i uh1
      s2[0] = fma_r(-cs, a0i, s2[0]);
      s2[1] = fma_r(cs, a0r, s2[1]);
      s3[0] = fma_r(cs, a1i, s3[0]);
      s3[1] = fma_r(-cs, a1r, s3[1]);
    } else {  // spin2 += SIG uh0, spin3 += SIG uh1
      s2[0] = fma_r(cs, a0r, s2[0]);
      s2[1] = fma_r(cs, a0i, s2[1]);
      s3[0] = fma_r(cs, a1r, s3[0]);
      s3[1] = fma_r(cs, a1i, s3[1]);
    }
  }
}

// o = U h (DAGGER = false) or U^+ h, for both spins of the half spinor; u row-major 3x3 complex.
// Written as explicit FMA chains: 12 instructions per complex output.
template <bool DAGGER, typename R>
__device__ __forceinline__ void su3_mul(const R* u, const R* h, R* o) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R re, im;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int e = DAGGER ? (b * 3 + a) : (a * 3 + b);
        const R ur = u[e * 2];
        const R ui = DAGGER ? -u[e * 2 + 1] : u[e * 2 + 1];
        const R hr = h[(sp * 3 + b) * 2], hi = h[(sp * 3 + b) * 2 + 1];
        if (b == 0) {
          re = ur * hr;
          im = ur * hi;
        } else {
          re = fma_r(ur, hr, re);
          im = fma_r(ur, hi, im);
        }
        re = fma_r(-ui, hi, re);
        im = fma_r(ui, hr, im);
      }
      o[(sp * 3 + a) * 2] = re;
      o[(sp * 3 + a) * 2 + 1] = im;
    }
}

// Third row of an SU(3) matrix from its first two: row2 = conj(row0 x row1).
template <typename R>
__device__ __forceinline__ void reconstruct_row2(R* u) {
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
    // row2[b] = conj(row0[b1] row1[b2] - row0[b2] row1[b1])
    const R xr = u[(0 * 3 + b1) * 2], xi = u[(0 * 3 + b1) * 2 + 1];
    const R yr = u[(1 * 3 + b2) * 2], yi = u[(1 * 3 + b2) * 2 + 1];
    const R zr = u[(0 * 3 + b2) * 2], zi = u[(0 * 3 + b2) * 2 + 1];
    const R wr = u[(1 * 3 + b1) * 2], wi = u[(1 * 3 + b1) * 2 + 1];
    const R cr = (xr * yr - xi * yi) - (zr * wr - zi * wi);
    const R ci = (xr * yi + xi * yr) - (zr * wi + zi * wr);
    u[(2 * 3 + b) * 2] = cr;
    u[(2 * 3 + b) * 2 + 1] = -ci;
  }
}

// Load one link (18 reals; the third row rebuilt as the conjugated cross product of the first
// two when only 12 are stored, which holds for every SU(3) matrix).
template <int P, bool C12>
__device__ __forceinline__ void load_link(const char* p, typename Store<P>::R* u) {
  using R = typename Store<P>::R;
  constexpr int VEC = Store<P>::VEC;
  constexpr int NR = C12 ? 12 : 18;
  constexpr int NV = (NR + VEC - 1) / VEC;
  R buf[NV * VEC];
#pragma unroll
  for (int v = 0; v < NV; ++v) ld16<P>(p + v * 16, buf + v * VEC);
#pragma unroll
  for (int i = 0; i < NR; ++i) u[i] = buf[i];
  if (C12) reconstruct_row2(u);
}

// A link from shared memory (plain loads; the staged kernel reads its own buffers).
template <int P, bool C12>
__device__ __forceinline__ void load_link_smem(const char* p, typename Store<P>::R* u) {
  using R = typename Store<P>::R;
  constexpr int VEC = Store<P>::VEC;
  constexpr int NR = C12 ? 12 : 18;
  constexpr int NV = (NR + VEC - 1) / VEC;
  R buf[NV * VEC];
#pragma unroll
  for (int v = 0; v < NV; ++v) ld16c<P>(p + v * 16, buf + v * VEC);
#pragma unroll
  for (int i = 0; i < NR; ++i) u[i] = buf[i];
  if (C12) reconstruct_row2(u);
}

// Copy one stored link (whole 16-byte vectors) from global to shared memory.
template <int P, bool C12>
__device__ __forceinline__ void copy_link(char* dst, const char* src) {
  constexpr int LB = link_bytes(sizeof(typename Store<P>::T), C12);
#pragma unroll
  for (int v = 0; v < LB / 16; ++v)
    *reinterpret_cast<uint4*>(dst + v * 16) = __ldg(reinterpret_cast<const uint4*>(src + v * 16));
}

// The direct kernel stages each site's eight links in shared memory once per CTA; every slice
// pair of the site then reads them from there. FP64 keeps the stored format (18 or 12 doubles per
// link). The packed kernels keep every link as 18 FP32 reals (80 bytes, converted from 16-bit
// storage and with the third row rebuilt once per site instead of once per thread), and pad each
// site's 640 bytes by 16: the four sites that one warp reads from then start 16 bytes apart
// modulo 128 and their 16-byte reads fall in different banks instead of four-way conflicts.
constexpr int DHOP_LINK_F32_BYTES = 80;
__host__ __device__ constexpr int dhop_link_site_bytes(int prec, bool c12) {
  return prec == P64 ? 8 * link_bytes(8, c12) : 8 * DHOP_LINK_F32_BYTES + 16;
}

// Shared memory of the staged links of one CTA, a multiple of 16 bytes.
__host__ __device__ constexpr size_t dhop_link_smem_bytes(int prec, int sites_per_cta, bool c12) {
  return (size_t)sites_per_cta * dhop_link_site_bytes(prec, c12);
}

// One link from global memory (any storage precision, 18 or 12 reals) to shared memory as 18
// FP32 reals.
template <int P, bool C12>
__device__ __forceinline__ void stage_link_f32(char* dst, const char* src) {
  float u[18];
  load_link<P, C12>(src, u);
  float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int v = 0; v < 4; ++v) d[v] = make_float4(u[4 * v], u[4 * v + 1], u[4 * v + 2], u[4 * v + 3]);
  reinterpret_cast<float2*>(dst)[8] = make_float2(u[16], u[17]);
}

__device__ __forceinline__ void load_link_f32(const char* s, float* u) {
  const float4* p = reinterpret_cast<const float4*>(s);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const float4 t = p[v];
    u[4 * v] = t.x;
    u[4 * v + 1] = t.y;
    u[4 * v + 2] = t.z;
    u[4 * v + 3] = t.w;
  }
  const float2 t = reinterpret_cast<const float2*>(s)[8];
  u[16] = t.x;
  u[17] = t.y;
}

// ---------------------------------------------------------------- packed two-slice algebra
// The same projection, SU(3) product and reconstruction on float2 values, .x for slice 2q and
// .y for slice 2q+1; every operation is one packed FP32x2 instruction.

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

template <int SIG>
__device__ __forceinline__ void project2(int mu, const float2* psi, float2* h) {
  const float2 P1 = f2((float)SIG), M1 = f2((float)-SIG);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float2 r0 = psi[(0 * 3 + c) * 2], i0 = psi[(0 * 3 + c) * 2 + 1];
    const float2 r1 = psi[(1 * 3 + c) * 2], i1 = psi[(1 * 3 + c) * 2 + 1];
    const float2 r2 = psi[(2 * 3 + c) * 2], i2 = psi[(2 * 3 + c) * 2 + 1];
    const float2 r3 = psi[(3 * 3 + c) * 2], i3 = psi[(3 * 3 + c) * 2 + 1];
    float2 h0r, h0i, h1r, h1i;
    if (mu == 0) {  // h0 = psi0 - SIG i psi3, h1 = psi1 - SIG i psi2
      h0r = ffma2(P1, i3, r0);
      h0i = ffma2(M1, r3, i0);
      h1r = ffma2(P1, i2, r1);
      h1i = ffma2(M1, r2, i1);
    } else if (mu == 1) {  // h0 = psi0 - SIG psi3, h1 = psi1 + SIG psi2
      h0r = ffma2(M1, r3, r0);
      h0i = ffma2(M1, i3, i0);
      h1r = ffma2(P1, r2, r1);
      h1i = ffma2(P1, i2, i1);
    } else if (mu == 2) {  // h0 = psi0 - SIG i psi2, h1 = psi1 + SIG i psi3
      h0r = ffma2(P1, i2, r0);
      h0i = ffma2(M1, r2, i0);
      h1r = ffma2(M1, i3, r1);
      h1i = ffma2(P1, r3, i1);
    } else {  // h0 = psi0 + SIG psi2, h1 = psi1 + SIG psi3
      h0r = ffma2(P1, r2, r0);
      h0i = ffma2(P1, i2, i0);
      h1r = ffma2(P1, r3, r1);
      h1i = ffma2(P1, i3, i1);
    }
    h[(0 * 3 + c) * 2] = h0r;
    h[(0 * 3 + c) * 2 + 1] = h0i;
    h[(1 * 3 + c) * 2] = h1r;
    h[(1 * 3 + c) * 2 + 1] = h1i;
  }
}

// o = U h or U^+ h for both spins of the half spinor and both slices; u scalar row-major 3x3.
template <bool DAGGER>
__device__ __forceinline__ void su3_mul2(const float* u, const float2* h, float2* o) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float2 re, im;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int e = DAGGER ? (b * 3 + a) : (a * 3 + b);
        const float ur = u[e * 2];
        const float ui = DAGGER ? -u[e * 2 + 1] : u[e * 2 + 1];
        const float2 hr = h[(sp * 3 + b) * 2], hi = h[(sp * 3 + b) * 2 + 1];
        if (b == 0) {
          re = fmul2(f2(ur), hr);
          im = fmul2(f2(ur), hi);
        } else {
          re = ffma2(f2(ur), hr, re);
          im = ffma2(f2(ur), hi, im);
        }
        re = ffma2(f2(-ui), hi, re);
        im = ffma2(f2(ui), hr, im);
      }
      o[(sp * 3 + a) * 2] = re;
      o[(sp * 3 + a) * 2 + 1] = im;
    }
}

// acc += c * reconstruct(uh), c = boundary phase times scale (the same for both slices).
template <int SIG>
__device__ __forceinline__ void accumulate2(int mu, const float2* uh, float c, float2* acc) {
  const float2 C = f2(c), CS = f2(SIG * c), MCS = f2(-SIG * c);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float2 a0r = uh[(0 * 3 + k) * 2], a0i = uh[(0 * 3 + k) * 2 + 1];
    const float2 a1r = uh[(1 * 3 + k) * 2], a1i = uh[(1 * 3 + k) * 2 + 1];
    float2* s0 = acc + (0 * 3 + k) * 2;
    float2* s1 = acc + (1 * 3 + k) * 2;
    float2* s2 = acc + (2 * 3 + k) * 2;
    float2* s3 = acc + (3 * 3 + k) * 2;
    s0[0] = ffma2(C, a0r, s0[0]);
    s0[1] = ffma2(C, a0i, s0[1]);
    s1[0] = ffma2(C, a1r, s1[0]);
    s1[1] = ffma2(C, a1i, s1[1]);
    if (mu == 0) {  // spin2 += SIG i uh1, spin3 += SIG i uh0
      s2[0] = ffma2(MCS, a1i, s2[0]);
      s2[1] = ffma2(CS, a1r, s2[1]);
      s3[0] = ffma2(MCS, a0i, s3[0]);
      s3[1] = ffma2(CS, a0r, s3[1]);
    } else if (mu == 1) {  // spin2 += SIG uh1, spin3 -= SIG uh0
      s2[0] = ffma2(CS, a1r, s2[0]);
      s2[1] = ffma2(CS, a1i, s2[1]);
      s3[0] = ffma2(MCS, a0r, s3[0]);
      s3[1] = ffma2(MCS, a0i, s3[1]);
    } else if (mu == 2) {  // spin2 += SIG i uh0, spin3 -= SIG i uh1
      s2[0] = ffma2(MCS, a0i, s2[0]);
      s2[1] = ffma2(CS, a0r, s2[1]);
      s3[0] = ffma2(CS, a1i, s3[0]);
      s3[1] = ffma2(MCS, a1r, s3[1]);
    } else {  // spin2 += SIG uh0, spin3 += SIG uh1
      s2[0] = ffma2(CS, a0r, s2[0]);
      s2[1] = ffma2(CS, a0i, s2[1]);
      s3[0] = ffma2(CS, a1r, s3[0]);
      s3[1] = ffma2(CS, a1i, s3[1]);
    }
  }
}

// ---------------------------------------------------------------- 16-bit storage projection
// With FP16/BF16 storage every element of the half spinor is a + s b (s = +-1) of two stored
// 16-bit values. Instead of widening both to FP32 and combining them with an FP32 FMA, the
// FP32 <- 16-bit mixed-precision instructions of sm_100 and later take b as it is stored:
// a is widened exactly (an FP32 add of -0, or for BF16 a shift into the upper half-word) and
// a + s b is then one FP32 operation with one rounding (s b is exact), so the result is
// bit-identical to widening both operands and computing in FP32, with half the conversions.
// Conversions run on a narrower pipe than FMAs on this part and were what bounded the 16-bit
// kernels.

template <int P>
__device__ __forceinline__ float widen16(unsigned short a) {
  if constexpr (P == P16) {
    float d;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(-0.0f));
    return d;
  } else {
    return __uint_as_float((uint32_t)a << 16);
  }
}

// a + S b in FP32 with one rounding; a already FP32, b a stored 16-bit value.
template <int P, int S>
__device__ __forceinline__ float add16(float a, unsigned short b) {
  float d;
  if constexpr (P == P16) {
    if constexpr (S > 0)
      asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(b), "f"(a));
    else
      asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(b), "h"((unsigned short)0xBC00), "f"(a));  // -1.0
  } else {
    if constexpr (S > 0)
      asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(b), "f"(a));
    else
      asm("fma.rn.f32.bf16 %0, %1, %2, %3;" : "=f"(d) : "h"(b), "h"((unsigned short)0xBF80), "f"(a));  // -1.0
  }
  return d;
}

// Both slices: word wa holds real a of slices (2q, 2q+1) as (low, high) 16-bit halves, wb real b.
template <int P, int S>
__device__ __forceinline__ float2 combine16(uint32_t wa, uint32_t wb) {
  unsigned short blo, bhi;
  asm("mov.b32 {%0, %1}, %2;" : "=h"(blo), "=h"(bhi) : "r"(wb));
  if constexpr (P == PB16) {
    // BF16 is the top half of an FP32 word: widen a in place (low half shifted up, high half
    // masked), one integer instruction each (measured 7% faster than unpacking it first)
    return make_float2(add16<P, S>(__uint_as_float(wa << 16), blo), add16<P, S>(__uint_as_float(wa & 0xffff0000u), bhi));
  } else {
    unsigned short alo, ahi;
    asm("mov.b32 {%0, %1}, %2;" : "=h"(alo), "=h"(ahi) : "r"(wa));
    return make_float2(add16<P, S>(widen16<P>(alo), blo), add16<P, S>(widen16<P>(ahi), bhi));
  }
}

// project2 on stored 16-bit words: w[r] holds real r of both slices of the pair.
template <int P, int SIG>
__device__ __forceinline__ void project2w(int mu, const uint32_t* w, float2* h) {
#define WR(sp, c) w[((sp)*3 + (c)) * 2]
#define WI(sp, c) w[((sp)*3 + (c)) * 2 + 1]
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float2 h0r, h0i, h1r, h1i;
    if (mu == 0) {  // h0 = psi0 - SIG i psi3, h1 = psi1 - SIG i psi2
      h0r = combine16<P, SIG>(WR(0, c), WI(3, c));
      h0i = combine16<P, -SIG>(WI(0, c), WR(3, c));
      h1r = combine16<P, SIG>(WR(1, c), WI(2, c));
      h1i = combine16<P, -SIG>(WI(1, c), WR(2, c));
    } else if (mu == 1) {  // h0 = psi0 - SIG psi3, h1 = psi1 + SIG psi2
      h0r = combine16<P, -SIG>(WR(0, c), WR(3, c));
      h0i = combine16<P, -SIG>(WI(0, c), WI(3, c));
      h1r = combine16<P, SIG>(WR(1, c), WR(2, c));
      h1i = combine16<P, SIG>(WI(1, c), WI(2, c));
    } else if (mu == 2) {  // h0 = psi0 - SIG i psi2, h1 = psi1 + SIG i psi3
      h0r = combine16<P, SIG>(WR(0, c), WI(2, c));
      h0i = combine16<P, -SIG>(WI(0, c), WR(2, c));
      h1r = combine16<P, -SIG>(WR(1, c), WI(3, c));
      h1i = combine16<P, SIG>(WI(1, c), WR(3, c));
    } else {  // h0 = psi0 + SIG psi2, h1 = psi1 + SIG psi3
      h0r = combine16<P, SIG>(WR(0, c), WR(2, c));
      h0i = combine16<P, SIG>(WI(0, c), WI(2, c));
      h1r = combine16<P, SIG>(WR(1, c), WR(3, c));
      h1i = combine16<P, SIG>(WI(1, c), WI(3, c));
    }
    h[(0 * 3 + c) * 2] = h0r;
    h[(0 * 3 + c) * 2 + 1] = h0i;
    h[(1 * 3 + c) * 2] = h1r;
    h[(1 * 3 + c) * 2 + 1] = h1i;
  }
#undef WR
#undef WI
}

// ---------------------------------------------------------------- layout accessors
// Site blocks are [chunk k][pair q] of 16-byte vectors (dwf_common.cuh). LSH > 0 fixes the
// number of pairs at compile time, so chunk offsets become immediates.

// Both slices of pair q as float2 (FP32 arithmetic; not for FP64). GLOBAL selects the
// read-only cache path (global memory) or plain loads (shared memory).
template <int P, int LSH, bool GLOBAL = true>
__device__ __forceinline__ void load_pair(const char* blk, int q, int Lsh_rt, float2* v) {
  constexpr int VEC = Store<P>::VEC, RV = Store<P>::RV, NCH = Store<P>::NCH;
  const int Lsh = LSH > 0 ? LSH : Lsh_rt;
  const char* b = blk + (size_t)q * 16;
#pragma unroll
  for (int k = 0; k < NCH; ++k) {
    float t[VEC];
    if (GLOBAL)
      ld16<P>(b + k * chunk_stride(Lsh), t);
    else
      ld16c<P>(b + k * chunk_stride(Lsh), t);
#pragma unroll
    for (int j = 0; j < RV; ++j) v[RV * k + j] = make_float2(t[2 * j], t[2 * j + 1]);
  }
}

// 16-bit storage: the 24 stored words of pair q (word r = real r of both slices), not widened.
template <int P, int LSH>
__device__ __forceinline__ void load_words(const char* blk, int q, int Lsh_rt, uint32_t* w) {
  static_assert(P == P16 || P == PB16, "16-bit storage only");
  const int Lsh = LSH > 0 ? LSH : Lsh_rt;
  const char* b = blk + (size_t)q * 16;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(b + k * chunk_stride(Lsh)));
    w[4 * k] = v.x;
    w[4 * k + 1] = v.y;
    w[4 * k + 2] = v.z;
    w[4 * k + 3] = v.w;
  }
}

template <int P, int LSH>
__device__ __forceinline__ void store_pair(char* blk, int q, int Lsh_rt, const float2* v) {
  constexpr int VEC = Store<P>::VEC, RV = Store<P>::RV, NCH = Store<P>::NCH;
  const int Lsh = LSH > 0 ? LSH : Lsh_rt;
  char* b = blk + (size_t)q * 16;
#pragma unroll
  for (int k = 0; k < NCH; ++k) {
    float t[VEC];
#pragma unroll
    for (int j = 0; j < RV; ++j) {
      t[2 * j] = v[RV * k + j].x;
      t[2 * j + 1] = v[RV * k + j].y;
    }
    st16<P>(b + k * chunk_stride(Lsh), t);
  }
}

// FP64: slice s alone; real k of slice s is the double at byte k * chunk_stride + s * 8.
template <int LSH, bool GLOBAL = true>
__device__ __forceinline__ void load_lane64(const char* blk, int s, int Lsh_rt, double* v) {
  const int Lsh = LSH > 0 ? LSH : Lsh_rt;
  const char* b = blk + (size_t)s * 8;
#pragma unroll
  for (int k = 0; k < 24; ++k) {
    const double* p = reinterpret_cast<const double*>(b + k * chunk_stride(Lsh));
    v[k] = GLOBAL ? __ldg(p) : *p;
  }
}

template <int LSH>
__device__ __forceinline__ void store_lane64(char* blk, int s, int Lsh_rt, const double* v) {
  const int Lsh = LSH > 0 ? LSH : Lsh_rt;
  char* b = blk + (size_t)s * 8;
#pragma unroll
  for (int k = 0; k < 24; ++k) *reinterpret_cast<double*>(b + k * chunk_stride(Lsh)) = v[k];
}

// Any precision: the 24 reals of slice s (the lane of its pair), in the arithmetic type.
template <int P, bool GLOBAL = true>
__device__ __forceinline__ void load_slice(const char* blk, int s, int Lsh, typename Store<P>::R* v) {
  if constexpr (P == P64) {
    load_lane64<0, GLOBAL>(blk, s, Lsh, v);
  } else {
    constexpr int VEC = Store<P>::VEC, RV = Store<P>::RV, NCH = Store<P>::NCH;
    const int l = s & 1;
    const char* b = blk + (size_t)(s >> 1) * 16;
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
      float t[VEC];
      if (GLOBAL)
        ld16<P>(b + k * chunk_stride(Lsh), t);
      else
        ld16c<P>(b + k * chunk_stride(Lsh), t);
#pragma unroll
      for (int j = 0; j < RV; ++j) v[RV * k + j] = t[2 * j + l];
    }
  }
}

// Packed precisions: reals r0 .. r0 + 11 (r0 = 0: the upper, P+ spins; 12: the lower) of slice s,
// widened to FP32.
template <int P>
__device__ __forceinline__ void load_slice_half(const char* blk, int s, int Lsh, int r0, float* v) {
  constexpr int VEC = Store<P>::VEC, RV = Store<P>::RV;
  const int l = s & 1;
  const char* b = blk + (size_t)(s >> 1) * 16;
#pragma unroll
  for (int k = 0; k < 12 / RV; ++k) {
    float t[VEC];
    ld16<P>(b + (r0 / RV + k) * chunk_stride(Lsh), t);
#pragma unroll
    for (int j = 0; j < RV; ++j) v[RV * k + j] = t[2 * j + l];
  }
}

// (Mooee aux)_s or (Mooee^+ aux)_s for one slice s < Ls (zero for the pad slice): the upper (P+)
// reals couple to s-1 and the lower (P-) reals to s+1, with +m replacing -1 on the wrap-around;
// the adjoint swaps them. GLOBAL = false reads a block staged in shared memory.
template <int P, bool DAG5, bool GLOBAL = true>
__device__ __forceinline__ void mooee_slice(const char* blk, int s, int Ls, int Lsh, double d5, double mass,
                                            typename Store<P>::R* o) {
  using R = typename Store<P>::R;
  if (s >= Ls) {
#pragma unroll
    for (int r = 0; r < 24; ++r) o[r] = 0;
    return;
  }
  const int sm = s > 0 ? s - 1 : Ls - 1;
  const int sp = s < Ls - 1 ? s + 1 : 0;
  const R cm = s > 0 ? R(-1) : R(mass);
  const R cp = s < Ls - 1 ? R(-1) : R(mass);
  const int s_up = DAG5 ? sp : sm, s_lo = DAG5 ? sm : sp;
  const R c_up = DAG5 ? cp : cm, c_lo = DAG5 ? cm : cp;
  const R d = R(d5);
  R self[24], up[24], lo[24];
  load_slice<P, GLOBAL>(blk, s, Lsh, self);
  load_slice<P, GLOBAL>(blk, s_up, Lsh, up);
  load_slice<P, GLOBAL>(blk, s_lo, Lsh, lo);
#pragma unroll
  for (int r = 0; r < 24; ++r) o[r] = d * self[r] + (r < 12 ? c_up * up[r] : c_lo * lo[r]);
}

// Shared-memory staging of the fifth-dimension inverse: the 24 reals of a slice, then the next
// slice INV_SLICE_STRIDE words (floats, doubles or float pairs) further. The stride is odd so that
// the threads of a warp, which store the same real of consecutive slices, hit different banks: with
// 24 the slices of a site were 48 or 96 words apart and a warp's stores fell on two banks (a
// 16-way conflict; at 24^4 x 12 the hop with the FP32 inverse took 180 us against 119 us for the
// plain hop, with 14.7 M bank conflicts).
constexpr int INV_SLICE_STRIDE = 25;

// In-place inverse of the fifth-dimension matrix along one real component of one site, held
// in shared memory with stride INV_SLICE_STRIDE between slices. FORWARD_FORM solves the chirality
// coupled to s-1: y_0 = (b_0 - m sum_{k>=1} d^-(Ls-k) b_k) / (d + m d^-(Ls-1)),
// y_s = (b_s + y_{s-1}) / d; otherwise the mirror image in s.
template <typename R, int S = INV_SLICE_STRIDE>
__device__ __forceinline__ void mooee_inv_line(R* v, int Ls, bool forward_form, R mass, R inv_d, R inv_den) {
  if (forward_form) {
    R acc = 0;
    for (int k = 1; k < Ls; ++k) acc = (acc + v[k * S]) * inv_d;
    R y = (v[0] - mass * acc) * inv_den;
    v[0] = y;
    for (int s = 1; s < Ls; ++s) {
      y = (v[s * S] + y) * inv_d;
      v[s * S] = y;
    }
  } else {
    R acc = 0;
    for (int k = Ls - 2; k >= 0; --k) acc = (acc + v[k * S]) * inv_d;
    R y = (v[(Ls - 1) * S] - mass * acc) * inv_den;
    v[(Ls - 1) * S] = y;
    for (int s = Ls - 2; s >= 0; --s) {
      y = (v[s * S] + y) * inv_d;
      v[s * S] = y;
    }
  }
}

// The packed kernels stage the inverse differently: per site 24 lines, one per real component,
// each holding the site's slices contiguously, so that a thread stores its two slices of a real
// as one float2 and a line moves with 128-bit accesses. A line is padded to an odd number of
// float4 (the eight lanes of a 128-bit access then cover all 32 banks), a site to a stride that
// puts consecutive sites' float2 stores on consecutive banks.
__host__ __device__ constexpr int inv_line_stride(int Ls) {
  return (((Ls + 3) / 4) & 1) ? ((Ls + 3) & ~3) : ((Ls + 3) & ~3) + 4;
}
__host__ __device__ constexpr int inv_site_stride(int Ls) {
  return 24 * inv_line_stride(Ls) +
         ((((2 * ls_half(Ls) + 3) & ~3) - 24 * inv_line_stride(Ls)) % 32 + 32) % 32;
}

// mooee_inv_line on one contiguous line of LS slices (compile-time), held in registers between
// one 128-bit load and one 128-bit store per four slices; the same operations in the same order.
template <int LS>
__device__ __forceinline__ void mooee_inv_line_vec(float* line, bool forward_form, float mass, float inv_d,
                                                   float inv_den) {
  constexpr int NV = (LS + 3) / 4;
  float v[4 * NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const float4 t = reinterpret_cast<const float4*>(line)[j];
    v[4 * j] = t.x;
    v[4 * j + 1] = t.y;
    v[4 * j + 2] = t.z;
    v[4 * j + 3] = t.w;
  }
  if (forward_form) {
    float acc = 0.f;
#pragma unroll
    for (int k = 1; k < LS; ++k) acc = (acc + v[k]) * inv_d;
    float y = (v[0] - mass * acc) * inv_den;
    v[0] = y;
#pragma unroll
    for (int s = 1; s < LS; ++s) {
      y = (v[s] + y) * inv_d;
      v[s] = y;
    }
  } else {
    float acc = 0.f;
#pragma unroll
    for (int k = LS - 2; k >= 0; --k) acc = (acc + v[k]) * inv_d;
    float y = (v[LS - 1] - mass * acc) * inv_den;
    v[LS - 1] = y;
#pragma unroll
    for (int s = LS - 2; s >= 0; --s) {
      y = (v[s] + y) * inv_d;
      v[s] = y;
    }
  }
#pragma unroll
  for (int j = 0; j < NV; ++j)
    reinterpret_cast<float4*>(line)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
}

// ---------------------------------------------------------------- kernel bodies

// Epilogue kinds compiled into a packed kernel: bit 0 the pre-operation (aux, Mooee aux, Mooee^+
// aux), bit 1 the post-operation (Mooee^-1, (Mooee^+)^-1). A launch runs the instantiation with
// exactly the parts it uses, so plain hops and single-epilogue hops keep fewer live registers.
//
// Two more bits serve the mixed-precision CG, which needs of Mpc^+ Mpc p only two numbers and one
// vector update (the Schur normal operator's launches 2 and 4, with their pre-operations):
//   EPI_NORM (4): store the result as usual and add |result|^2 (the squared norm of Mpc p, which
//                 equals p^+ Mpc^+ Mpc p) to the launch's per-CTA partial sums;
//   EPI_AXPY (8): do not store the result; update the FP32 field r -= c * result with c read from
//                 device memory (the CG step length), and add |r|^2 to the partial sums.
// Neither is combined with a post-operation; EPI_NORM also serves full-lattice launches (one
// partial per CTA of either half), EPI_AXPY only half-lattice ones.
//   EPI_HALO (16): the lattice is one block of a lattice split in t (see DhopArgs): hops that leave
//                 the block in t take the neighbours' projected faces; launched over the face
//                 planes only (the interior needs no halo and runs the plain instantiation).
enum EpiKind : int { EPI_NONE = 0, EPI_PRE = 1, EPI_POST = 2, EPI_BOTH = 3, EPI_NORM = 4, EPI_AXPY = 8, EPI_HALO = 16 };

// Sum of one value per thread over the CTA in a fixed order (warp shuffles, then the warps in
// order), written by thread 0 to *dst.
__device__ __forceinline__ void cta_sum_to(double v, double* dst) {
  __shared__ double wsum[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) wsum[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += wsum[w];
    *dst = t;
  }
}

// FP32 / FP16 / BF16: one thread per (site, slice pair), packed two-wide arithmetic.
template <int P, bool DAG, bool C12, int LSC, int EK>
__device__ __forceinline__ void dhop_body_pair(const DhopArgs& a) {
  using T = typename Store<P>::T;
  constexpr int LB = link_bytes(sizeof(T), C12);
  constexpr int SF = DAG ? +1 : -1;  // forward projector (1 + SF gamma)
  constexpr int SB = -SF;            // backward projector
  constexpr int LSHC = LSC > 0 ? ls_half(LSC) : 0;
  const int Ls = LSC > 0 ? LSC : a.g.Ls;
  const int Lsh = LSC > 0 ? LSHC : ls_half(a.g.Ls);
  const int tid = threadIdx.x;
  const int site_local = tid / Lsh;
  const int q = tid - site_local * Lsh;
  // Every CTA of a launch is full: the launcher covers a ragged end of the lattice with a second,
  // one-CTA launch whose site_base places it flush with the end (it rewrites a few sites with the
  // same values). The kernel then has no tail handling at all: a per-thread guard around the hop
  // loop, or a clamped site index, measured 5-10% slower.
  // the other half of a full-lattice launch: CTAs [blocks1, 2 blocks1), or, with interleave,
  // the odd CTAs (the halves then read the same links at about the same time)
  const bool second = a.interleave ? ((int)blockIdx.x & 1) != 0 : (int)blockIdx.x >= a.blocks1;
  const int bid = a.interleave ? (int)blockIdx.x >> 1 : second ? (int)blockIdx.x - a.blocks1 : (int)blockIdx.x;
  const int out_parity = second ? 1 - a.out_parity : a.out_parity;
  int cta = bid;
  if (a.zblk > 0) {  // plane w = zi + zblk * (t + Lt * zb) of the walk is the lattice's plane z + Lz * t
    const uint32_t w = fdiv((uint32_t)bid, a.div_cpp);
    const int in_plane = bid - (int)w * a.ctas_per_plane;
    const uint32_t r = fdiv(w, a.div_zblk);
    const int zi = (int)(w - r * (uint32_t)a.zblk);
    const uint32_t zb = fdiv(r, a.div_lt);
    const int t = (int)(r - zb * (uint32_t)a.g.L[3]);
    cta = in_plane + a.ctas_per_plane * ((int)zb * a.zblk + zi + a.g.L[2] * t);
  }
  const int site = a.site_base + cta * a.sites_per_cta + site_local;
  constexpr bool active = true;
  const size_t site_bytes = (size_t)Lsh * 2 * 24 * sizeof(T);
  const float alpha = (float)a.alpha;

  float2 acc[24];
#pragma unroll
  for (int r = 0; r < 24; ++r) acc[r] = make_float2(0.f, 0.f);

  // The eight links of each site, staged once per CTA as FP32: thread q of a site fetches the
  // links of hops q, q + Lsh, ... (hop h = 2 mu + backward), so every link is requested from
  // memory once instead of once per slice pair; the hops then read them from shared memory.
  constexpr int LSS = dhop_link_site_bytes(P, false);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  char* lsm = reinterpret_cast<char*>(smem_raw) + (size_t)site_local * LSS;  // [hop 8][80 bytes]
  const char* Uo = static_cast<const char*>(second ? a.Uin : a.Uout);  // links of the output parity
  const char* Ui = static_cast<const char*>(second ? a.Uout : a.Uin);
  // Neighbour indices and boundary phases of the eight hops, all computed before the first load
  // so that the hop loop below is straight-line code whose loads the compiler can issue early.
  int nb[8], phs[8];
  bool edge_lo = false, edge_hi = false;  // EPI_HALO: first / last t-plane of the block
  {
    int c[4];
    cb_coords(a.g, site, out_parity, c);
#pragma unroll
    for (int h = 0; h < 8; ++h) nb[h] = cb_neighbour(a.g, site, c, h >> 1, (h & 1) == 0, phs[h]);
    if constexpr ((EK & EPI_HALO) != 0) {
      edge_lo = c[3] == 0;
      edge_hi = c[3] == a.g.L[3] - 1;
    }
    // Launched as a programmatic dependent of the previous kernel on the stream, the CTA may start
    // before that kernel has finished: everything above reads only the launch arguments; wait for
    // the previous grid (its writes visible) before the first load of memory it may have written,
    // the links included (they are packed lazily by a kernel that can precede this one). Without
    // a dependency this returns at once.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int h = q; h < 8; h += Lsh) {
      const int mu = h >> 1;
      const char* src = (h & 1) == 0 ? Uo + ((size_t)site * 4 + mu) * LB : Ui + ((size_t)nb[h] * 4 + mu) * LB;
      if ((EK & EPI_HALO) != 0 && h == 7 && edge_lo)  // U_t(x - t) lives on the previous block
        src = static_cast<const char*>(a.halo_links) + (size_t)site * LB;
      stage_link_f32<P, C12>(lsm + h * DHOP_LINK_F32_BYTES, src);
    }
  }
  __syncthreads();

  {
    const char* in = static_cast<const char*>(second ? a.in2 : a.in);
#pragma unroll
    for (int hop = 0; hop < 8; ++hop) {
      // hop = 2 mu: forward, (1 + SF gamma_mu) U_mu(x) psi(x + mu);
      // hop = 2 mu + 1: backward, (1 + SB gamma_mu) U_mu(x - mu)^+ psi(x - mu).
      // The neighbour's vectors are requested first, the link is read from shared memory after.
      const int mu = hop >> 1;
      const bool fwd = (hop & 1) == 0;
      float2 h[12], uh[12];
      float u[18];
      const char* nbp = in + site_offset(nb[hop], Lsh, site_bytes);
      bool from_halo = false;
      if constexpr ((EK & EPI_HALO) != 0) from_halo = (hop == 6 && edge_hi) || (hop == 7 && edge_lo);
      if (from_halo) {
        // the neighbour block's projected half spinor, already multiplied by any boundary phase
        const int f = hop == 6 ? site - (a.g.N4h - a.plane) : site;
        const float4* hp = static_cast<const float4*>(hop == 6 ? a.halo_fwd : a.halo_bwd) + (size_t)f * 6 * Lsh + q;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          const float4 t = __ldg(hp + (size_t)j * Lsh);
          h[2 * j] = make_float2(t.x, t.y);
          h[2 * j + 1] = make_float2(t.z, t.w);
        }
        load_link_f32(lsm + hop * DHOP_LINK_F32_BYTES, u);
      } else if constexpr (P == P32) {
        float2 psi[24];
        load_pair<P, LSHC>(nbp, q, Lsh, psi);
        load_link_f32(lsm + hop * DHOP_LINK_F32_BYTES, u);
        if (fwd)
          project2<SF>(mu, psi, h);
        else
          project2<SB>(mu, psi, h);
      } else {
        uint32_t w[24];
        load_words<P, LSHC>(nbp, q, Lsh, w);
        load_link_f32(lsm + hop * DHOP_LINK_F32_BYTES, u);
        if (fwd)
          project2w<P, SF>(mu, w, h);
        else
          project2w<P, SB>(mu, w, h);
      }
      const float cph = (!from_halo && phs[hop] < 0) ? -alpha : alpha;
      if (fwd) {
        su3_mul2<false>(u, h, uh);
        accumulate2<SF>(mu, uh, cph, acc);
      } else {
        su3_mul2<true>(u, h, uh);
        accumulate2<SB>(mu, uh, cph, acc);
      }
    }
  }

  // The next kernel on the stream may be scheduled once every CTA has passed this point (it then
  // waits at its own griddepcontrol.wait for this grid to finish); without one this does nothing.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  // ------------------------------------------------------------ epilogue
  char* outb = static_cast<char*>(second ? a.out2 : a.out) + site_offset(site, Lsh, site_bytes);
  if ((EK & EPI_PRE) && active && a.pre != PRE_NONE) {
    const char* auxb = static_cast<const char*>(second ? a.aux2 : a.aux) + site_offset(site, Lsh, site_bytes);
    const float2 B = f2((float)a.beta);
    if (a.pre == PRE_AUX) {
      float2 o[24];
      load_pair<P, LSHC>(auxb, q, Lsh, o);
#pragma unroll
      for (int r = 0; r < 24; ++r) acc[r] = ffma2(B, o[r], acc[r]);
    } else {
      // beta (Mooee aux)_s = beta ((5 - M5) aux_s + c_up aux_{s_up}[upper] + c_lo aux_{s_lo}[lower]):
      // the pair's own slices once, then only the 12-real half of each coupled neighbour slice.
      const bool dag5 = a.pre == PRE_MOOEE_DAG;
      const float beta = (float)a.beta, mass = (float)a.mass;
      float2 own[24];
      load_pair<P, LSHC>(auxb, q, Lsh, own);
      const float2 BD = f2(beta * (float)a.d5);
#pragma unroll
      for (int r = 0; r < 24; ++r) acc[r] = ffma2(BD, own[r], acc[r]);
#pragma unroll
      for (int l = 0; l < 2; ++l) {
        const int s = 2 * q + l;
        if (s >= Ls) continue;  // the zero pad slice
        const int sm = s > 0 ? s - 1 : Ls - 1, sp = s < Ls - 1 ? s + 1 : 0;
        const float cm = s > 0 ? -1.f : mass, cp = s < Ls - 1 ? -1.f : mass;
        const int s_up = dag5 ? sp : sm, s_lo = dag5 ? sm : sp;
        const float c_up = beta * (dag5 ? cp : cm), c_lo = beta * (dag5 ? cm : cp);
        float x[12];
        load_slice_half<P>(auxb, s_up, Lsh, 0, x);
#pragma unroll
        for (int r = 0; r < 12; ++r) {
          if (l == 0)
            acc[r].x = fmaf(c_up, x[r], acc[r].x);
          else
            acc[r].y = fmaf(c_up, x[r], acc[r].y);
        }
        load_slice_half<P>(auxb, s_lo, Lsh, 12, x);
#pragma unroll
        for (int r = 0; r < 12; ++r) {
          if (l == 0)
            acc[12 + r].x = fmaf(c_lo, x[r], acc[12 + r].x);
          else
            acc[12 + r].y = fmaf(c_lo, x[r], acc[12 + r].y);
        }
      }
    }
  }
  const bool pad_lane = (Ls & 1) && q == Lsh - 1;  // slice 2q+1 is the zero pad
  if (!(EK & EPI_POST) || a.post == POST_NONE) {
    if (pad_lane) {
#pragma unroll
      for (int r = 0; r < 24; ++r) acc[r].y = 0.f;
    }
    if constexpr ((EK & (EPI_NORM | EPI_AXPY)) != 0) {
      const bool owned = site >= a.own_from;
      float n2 = 0.f;
      if constexpr ((EK & EPI_AXPY) != 0) {
        // r -= c * result (FP32 field, the same site blocks with FP32 vectors)
        char* rb = reinterpret_cast<char*>(a.r) + site_offset(site, Lsh, (size_t)Lsh * 2 * 24 * sizeof(float));
        float2 rv[24];
        load_pair<P32, LSHC>(rb, q, Lsh, rv);
        const float2 MC = f2(-(float)*a.axpy_coef);
#pragma unroll
        for (int r = 0; r < 24; ++r) {
          rv[r] = ffma2(MC, acc[r], rv[r]);
          n2 = fmaf(rv[r].x, rv[r].x, fmaf(rv[r].y, rv[r].y, n2));
        }
        if (owned) store_pair<P32, LSHC>(rb, q, Lsh, rv);
      } else {
        store_pair<P, LSHC>(outb, q, Lsh, acc);
#pragma unroll
        for (int r = 0; r < 24; ++r) n2 = fmaf(acc[r].x, acc[r].x, fmaf(acc[r].y, acc[r].y, n2));
      }
      cta_sum_to(owned ? (double)n2 : 0.0, a.red + a.red_base + (int)blockIdx.x);
    } else {
      store_pair<P, LSHC>(outb, q, Lsh, acc);
    }
    return;
  }
  // Fifth-dimension inverse through shared memory (after the staged links): whole sites live in
  // this CTA, staged as lines (inv_site_stride / inv_line_stride; the pad slice of an odd Ls is
  // stored past the line's end and never read).
  float* sm = reinterpret_cast<float*>(smem_raw + dhop_link_smem_bytes(P, a.sites_per_cta, false));
  const int lst = inv_line_stride(Ls), sst = inv_site_stride(Ls);
  if (active) {
    float* d0 = sm + (size_t)site_local * sst + 2 * q;
#pragma unroll
    for (int r = 0; r < 24; ++r) *reinterpret_cast<float2*>(d0 + r * lst) = acc[r];
  }
  __syncthreads();
  const int nsites = a.sites_per_cta;
  for (int task = tid; task < nsites * 24; task += blockDim.x) {
    const int sl = task / 24;
    const int r = task - sl * 24;
    const bool upper = r < 12;
    const bool forward_form = (a.post == POST_INV) ? upper : !upper;
    float* line = sm + (size_t)sl * sst + r * lst;
    if constexpr (LSC > 0)
      mooee_inv_line_vec<LSC>(line, forward_form, (float)a.mass, (float)a.inv_d5, (float)a.inv_den);
    else
      mooee_inv_line<float, 1>(line, Ls, forward_form, (float)a.mass, (float)a.inv_d5, (float)a.inv_den);
  }
  __syncthreads();
  if (active) {
    const float* s0 = sm + (size_t)site_local * sst + 2 * q;
#pragma unroll
    for (int r = 0; r < 24; ++r) {
      const float2 v = *reinterpret_cast<const float2*>(s0 + r * lst);
      acc[r] = make_float2(v.x, pad_lane ? 0.f : v.y);
    }
    store_pair<P, LSHC>(outb, q, Lsh, acc);
  }
}

// FP64: one thread per (site, slice), scalar arithmetic.
template <bool DAG, bool C12, int LSC>
__device__ __forceinline__ void dhop_body_lane64(const DhopArgs& a) {
  constexpr int LB = link_bytes(8, C12);
  constexpr int SF = DAG ? +1 : -1;
  constexpr int SB = -SF;
  constexpr int LSHC = LSC > 0 ? ls_half(LSC) : 0;
  const int Ls = LSC > 0 ? LSC : a.g.Ls;
  const int Lsh = LSC > 0 ? LSHC : ls_half(a.g.Ls);
  const int Lsp = 2 * Lsh;
  const int tid = threadIdx.x;
  const int site_local = tid / Lsp;
  const int s = tid - site_local * Lsp;
  const int site = blockIdx.x * a.sites_per_cta + site_local;
  const bool active = site_local < a.sites_per_cta && site < a.g.N4h;
  const size_t site_bytes = (size_t)Lsp * 24 * 8;
  const double alpha = a.alpha;

  double acc[24];
#pragma unroll
  for (int r = 0; r < 24; ++r) acc[r] = 0;
  // links staged once per CTA, as in dhop_body_pair
  extern __shared__ __align__(16) unsigned char smem_raw[];
  char* lsm = reinterpret_cast<char*>(smem_raw);  // [site_local][hop 8][LB]
  int c[4];
  if (active) {
    cb_coords(a.g, site, a.out_parity, c);
    const char* Uo = static_cast<const char*>(a.Uout);
    const char* Ui = static_cast<const char*>(a.Uin);
    for (int h = s; h < 8; h += Lsp) {
      const int mu = h >> 1;
      const char* src;
      if ((h & 1) == 0) {
        src = Uo + ((size_t)site * 4 + mu) * LB;
      } else {
        int ph;
        src = Ui + ((size_t)cb_neighbour(a.g, site, c, mu, false, ph) * 4 + mu) * LB;
      }
      copy_link<P64, C12>(lsm + ((size_t)site_local * 8 + h) * LB, src);
    }
  }
  __syncthreads();
  if (active) {
    const char* in = static_cast<const char*>(a.in);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      {
        int ph;
        const int j = cb_neighbour(a.g, site, c, mu, true, ph);
        double u[18], psi[24], h[12], uh[12];
        load_link_smem<P64, C12>(lsm + ((size_t)site_local * 8 + 2 * mu) * LB, u);
        load_lane64<LSHC>(in + site_offset(j, Lsh, site_bytes), s, Lsh, psi);
        project<SF>(mu, psi, h);
        su3_mul<false>(u, h, uh);
        accumulate<SF>(mu, uh, ph < 0 ? -alpha : alpha, acc);
      }
      {
        int ph;
        const int j = cb_neighbour(a.g, site, c, mu, false, ph);
        double u[18], psi[24], h[12], uh[12];
        load_link_smem<P64, C12>(lsm + ((size_t)site_local * 8 + 2 * mu + 1) * LB, u);
        load_lane64<LSHC>(in + site_offset(j, Lsh, site_bytes), s, Lsh, psi);
        project<SB>(mu, psi, h);
        su3_mul<true>(u, h, uh);
        accumulate<SB>(mu, uh, ph < 0 ? -alpha : alpha, acc);
      }
    }
  }
  char* outb = static_cast<char*>(a.out) + site_offset(site, Lsh, site_bytes);
  if (active && a.pre != PRE_NONE) {
    const char* auxb = static_cast<const char*>(a.aux) + site_offset(site, Lsh, site_bytes);
    double o[24];
    if (a.pre == PRE_AUX)
      load_lane64<LSHC>(auxb, s, Lsh, o);
    else if (a.pre == PRE_MOOEE)
      mooee_slice<P64, false>(auxb, s, Ls, Lsh, a.d5, a.mass, o);
    else
      mooee_slice<P64, true>(auxb, s, Ls, Lsh, a.d5, a.mass, o);
#pragma unroll
    for (int r = 0; r < 24; ++r) acc[r] = fma(a.beta, o[r], acc[r]);
  }
  const bool pad = s >= Ls;
  if (a.post == POST_NONE) {
    if (active) {
      if (pad) {
#pragma unroll
        for (int r = 0; r < 24; ++r) acc[r] = 0;
      }
      store_lane64<LSHC>(outb, s, Lsh, acc);
    }
    return;
  }
  double* sm = reinterpret_cast<double*>(smem_raw + dhop_link_smem_bytes(P64, a.sites_per_cta, C12));
  if (active && !pad) {
    double* dst = sm + ((size_t)site_local * Ls + s) * INV_SLICE_STRIDE;
#pragma unroll
    for (int r = 0; r < 24; ++r) dst[r] = acc[r];
  }
  __syncthreads();
  const int first_site = blockIdx.x * a.sites_per_cta;
  const int nsites = min(a.sites_per_cta, a.g.N4h - first_site);
  for (int task = tid; task < nsites * 24; task += blockDim.x) {
    const int sl = task / 24;
    const int r = task - sl * 24;
    const bool upper = r < 12;
    const bool forward_form = (a.post == POST_INV) ? upper : !upper;
    mooee_inv_line<double>(sm + (size_t)sl * Ls * INV_SLICE_STRIDE + r, Ls, forward_form, a.mass, a.inv_d5,
                           a.inv_den);
  }
  __syncthreads();
  if (active) {
    if (!pad) {
      const double* src = sm + ((size_t)site_local * Ls + s) * INV_SLICE_STRIDE;
#pragma unroll
      for (int r = 0; r < 24; ++r) acc[r] = src[r];
    } else {
#pragma unroll
      for (int r = 0; r < 24; ++r) acc[r] = 0;
    }
    store_lane64<LSHC>(outb, s, Lsh, acc);
  }
}

// Register budget. Every launch of dhop_kernel has at most 128 threads (128 / threads-per-site
// whole sites). The packed kernels keep four such CTAs per SM (128 registers per thread, no
// spills; measured against three CTAs with 156-168 registers: FP16 storage 43.1 -> 41.0 us at
// 16^4 x 16 and 633 -> 586 us at 32^4 x 16, FP32 and BF16 within 1-2%); the FP64 kernel is
// bound by the FP64 pipe and keeps more registers instead.
template <int P>
struct DhopOccupancy {
  static constexpr int THREADS = 128;
  static constexpr int MIN_BLOCKS = (P == P64) ? 1 : 4;
};

// Threads per site: slice pairs (packed kernels) or padded slices (FP64).
inline int dhop_threads_per_site(int prec, int Ls) { return prec == P64 ? ls_padded(Ls) : ls_half(Ls); }

// Ls values with a compile-time specialisation; any other Ls runs the generic kernel (LSC = 0).
#define DWF_LS_SPECIALISATIONS(M) M(8) M(12) M(16)
inline bool dhop_ls_specialised(int Ls) { return Ls == 8 || Ls == 12 || Ls == 16; }

// C12 selects the stored link format; EK the epilogue kind (EPI_BOTH for FP64).
template <int P, bool DAG, bool C12, int LSC, int EK>
__global__ void __launch_bounds__(DhopOccupancy<P>::THREADS, DhopOccupancy<P>::MIN_BLOCKS) dhop_kernel(const __grid_constant__ DhopArgs a) {
  if constexpr (P == P64)
    dhop_body_lane64<DAG, C12, LSC>(a);
  else
    dhop_body_pair<P, DAG, C12, LSC, EK>(a);
}

// Host-side launcher, instantiated once per storage precision in its own translation unit.
template <int P>
cudaError_t launch_dhop(const DhopArgs& a, bool dag, bool c12, int threads, int blocks, size_t smem,
                        cudaStream_t stream);
template <>
cudaError_t launch_dhop<P64>(const DhopArgs&, bool, bool, int, int, size_t, cudaStream_t);
template <>
cudaError_t launch_dhop<P32>(const DhopArgs&, bool, bool, int, int, size_t, cudaStream_t);
template <>
cudaError_t launch_dhop<P16>(const DhopArgs&, bool, bool, int, int, size_t, cudaStream_t);
template <>
cudaError_t launch_dhop<PB16>(const DhopArgs&, bool, bool, int, int, size_t, cudaStream_t);

}  // namespace gdwf
