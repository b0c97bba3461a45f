// Shared device-side definitions of the GB300 domain-wall operator library: storage
// precisions, the device field layout, fast integer division and lattice geometry.
//
// Device spinor layout (one checkerboard half of a 5D field). The fifth dimension is padded to
// an even length Lsp = Ls + (Ls & 1) (the pad slice, if any, is always zero) and handled in
// slice pairs (2q, 2q+1), q < Lsh = Lsp / 2. The Lsp x 24 reals of a 4D checkerboard site i (cb
// index = lexicographic 4D index / 2, x fastest) are 16-byte vectors indexed [chunk k][pair q]:
// vector (k, q) holds reals RV*k .. RV*k + RV - 1 of both slices of pair q, real-major: value
// 2j + l is real RV*k + j of slice 2q + l. RV = 1 (FP64), 2 (FP32), 4 (FP16/BF16); NCH = 24 / RV.
// Sites are stored in blocks of SITE_BLOCK = 4 consecutive cb sites: within a block, chunk k holds
// the four sites' Lsh vectors of that chunk one after another ([block][chunk k][site r][pair q]),
// so vector (k, q) of site i is at byte
//   site_offset(i) + k * chunk_stride + q * 16,
//   site_offset(i) = (i / 4) * 4 * site_bytes + (i % 4) * Lsh * 16,  chunk_stride = 4 * Lsh * 16,
// with site_bytes = Lsh * 2 * 24 * real_bytes. Why blocks: the threads of a warp read chunk k for
// whole sites, and a site's chunk is Lsh * 16 bytes (96 for Ls = 12); grouping four sites makes
// each warp load a run of whole 128-byte lines for any Ls (measured: the Ls = 12 hopping kernel
// 20% faster). Why pairs: with one thread per (site, pair), every real arrives as the two slices'
// values side by side, so the FP32 arithmetic runs as packed two-wide instructions (one
// instruction per two slices) and each link is loaded once for two slices. In FP64 the same
// bytes read as [real k][slice s] with stride chunk_stride between reals. Every half field holds
// a whole number of blocks (V / 2 is a multiple of 8 for even extents).
//
// A full field is the even half followed by the odd half.
//
// Device gauge layout, per parity p: [cb site][mu 0..3][link], each link the row-major 3x3
// complex matrix U_mu(x) (18 reals) or, compressed, its first two rows (12 reals), padded to a
// multiple of 16 bytes so that it is loaded as whole 16-byte vectors.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gdwf {

enum Prec : int { P64 = 0, P32 = 1, P16 = 2, PB16 = 3 };

// T: storage type; R: arithmetic type; VEC: values per 16-byte vector; RV = VEC / 2 reals (of
// two slices) per vector; NCH = 24 / RV vectors per slice pair.
template <int P>
struct Store;
template <>
struct Store<P64> {
  using T = double;
  using R = double;
  static constexpr int VEC = 2;
  static constexpr int RV = 1;
  static constexpr int NCH = 24;
};
template <>
struct Store<P32> {
  using T = float;
  using R = float;
  static constexpr int VEC = 4;
  static constexpr int RV = 2;
  static constexpr int NCH = 12;
};
template <>
struct Store<P16> {
  using T = __half;
  using R = float;
  static constexpr int VEC = 8;
  static constexpr int RV = 4;
  static constexpr int NCH = 6;
};
template <>
struct Store<PB16> {
  using T = __nv_bfloat16;
  using R = float;
  static constexpr int VEC = 8;
  static constexpr int RV = 4;
  static constexpr int NCH = 6;
};

inline int prec_bytes(int p) { return p == P64 ? 8 : p == P32 ? 4 : 2; }
inline int prec_vec(int p) { return 16 / prec_bytes(p); }

// Slice pairs per site and the padded fifth-dimension extent.
__host__ __device__ constexpr int ls_half(int Ls) { return (Ls + 1) >> 1; }
__host__ __device__ constexpr int ls_padded(int Ls) { return 2 * ls_half(Ls); }

// Site blocks of the device layout (see above).
constexpr int SITE_BLOCK = 4;
__host__ __device__ constexpr size_t chunk_stride(int Lsh) { return (size_t)SITE_BLOCK * Lsh * 16; }
__host__ __device__ inline size_t site_offset(long i, int Lsh, size_t site_bytes) {
  return (size_t)(i >> 2) * SITE_BLOCK * site_bytes + (size_t)(i & 3) * Lsh * 16;
}

// Bytes of one stored link (18 or 12 reals) rounded up to 16.
__host__ __device__ constexpr int link_bytes(int real_bytes, bool c12) {
  return (((c12 ? 12 : 18) * real_bytes) + 15) / 16 * 16;
}

// ---------------------------------------------------------------- 16-byte vector loads/stores

// Read-only input: non-coherent global load, the 16 bytes at p as VEC reals.
template <int P>
__device__ __forceinline__ void ld16(const void* p, typename Store<P>::R* r);

template <>
__device__ __forceinline__ void ld16<P64>(const void* p, double* r) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  r[0] = v.x;
  r[1] = v.y;
}
template <>
__device__ __forceinline__ void ld16<P32>(const void* p, float* r) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  r[0] = v.x;
  r[1] = v.y;
  r[2] = v.z;
  r[3] = v.w;
}
template <>
__device__ __forceinline__ void ld16<P16>(const void* p, float* r) {
  const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __half2 h;
    memcpy(&h, &w[i], 4);
    const float2 f = __half22float2(h);
    r[2 * i] = f.x;
    r[2 * i + 1] = f.y;
  }
}
template <>
__device__ __forceinline__ void ld16<PB16>(const void* p, float* r) {
  const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __nv_bfloat162 h;
    memcpy(&h, &w[i], 4);
    const float2 f = __bfloat1622float2(h);
    r[2 * i] = f.x;
    r[2 * i + 1] = f.y;
  }
}

// Coherent load, for buffers that the same launch also writes (read-modify-write updates).
template <int P>
__device__ __forceinline__ void ld16c(const void* p, typename Store<P>::R* r) {
  const uint4 v = *reinterpret_cast<const uint4*>(p);
  if constexpr (P == P64) {
    double2 d;
    memcpy(&d, &v, 16);
    r[0] = d.x;
    r[1] = d.y;
  } else if constexpr (P == P32) {
    float4 f;
    memcpy(&f, &v, 16);
    r[0] = f.x;
    r[1] = f.y;
    r[2] = f.z;
    r[3] = f.w;
  } else {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 f;
      if constexpr (P == P16) {
        __half2 h;
        memcpy(&h, &w[i], 4);
        f = __half22float2(h);
      } else {
        __nv_bfloat162 h;
        memcpy(&h, &w[i], 4);
        f = __bfloat1622float2(h);
      }
      r[2 * i] = f.x;
      r[2 * i + 1] = f.y;
    }
  }
}

template <int P>
__device__ __forceinline__ void st16(void* p, const typename Store<P>::R* r);

template <>
__device__ __forceinline__ void st16<P64>(void* p, const double* r) {
  *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]);
}
template <>
__device__ __forceinline__ void st16<P32>(void* p, const float* r) {
  *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
}
template <>
__device__ __forceinline__ void st16<P16>(void* p, const float* r) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __half2 h = __floats2half2_rn(r[2 * i], r[2 * i + 1]);
    memcpy(&w[i], &h, 4);
  }
  *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}
template <>
__device__ __forceinline__ void st16<PB16>(void* p, const float* r) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(r[2 * i], r[2 * i + 1]);
    memcpy(&w[i], &h, 4);
  }
  *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}

// Store 16 bytes converted straight from FP64 values (one rounding to the storage format).
template <int P>
__device__ __forceinline__ void st16d(void* p, const double* v) {
  if constexpr (P == P64) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  } else if constexpr (P == P32) {
    *reinterpret_cast<float4*>(p) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
  } else {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint16_t lo, hi;
      if constexpr (P == P16) {
        const __half a = __double2half(v[2 * i]), b = __double2half(v[2 * i + 1]);
        memcpy(&lo, &a, 2);
        memcpy(&hi, &b, 2);
      } else {
        const __nv_bfloat16 a = __double2bfloat16(v[2 * i]), b = __double2bfloat16(v[2 * i + 1]);
        memcpy(&lo, &a, 2);
        memcpy(&hi, &b, 2);
      }
      w[i] = (uint32_t)lo | ((uint32_t)hi << 16);
    }
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// ---------------------------------------------------------------- fast division

// Division by a run-time invariant d (Granlund & Montgomery, PLDI 1994): with
// l = ceil(log2 d) and m = ceil(2^(32+l) / d), q = floor(n m / 2^(32+l)) for all n < 2^31.
struct FastDiv {
  uint64_t m;
  uint32_t shift;
  uint32_t d;
};

inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  FastDiv f;
  f.d = d;
  f.shift = 32 + l;
  f.m = ((1ull << (32 + l)) + d - 1) / d;
  return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  return (uint32_t)(((uint64_t)n * f.m) >> f.shift);
}

// ---------------------------------------------------------------- geometry

struct Geom {
  int L[4];        // Lx, Ly, Lz, Lt (all even)
  int Lxh;         // Lx / 2
  int Ls;          // fifth-dimension extent
  int N4h;         // V / 2, checkerboard sites per parity
  int stride[4];   // cb-index steps for x (unused), y, z, t hops: Lxh, Lxh*Ly, Lxh*Ly*Lz
  int bc[4];       // +1 periodic, -1 antiperiodic, per direction
  FastDiv div_lxh, div_ly, div_lz;
};

// 4D coordinates of checkerboard site i of parity p.
__device__ __forceinline__ void cb_coords(const Geom& g, int i, int p, int c[4]) {
  const uint32_t r0 = fdiv((uint32_t)i, g.div_lxh);
  const int xh = i - (int)r0 * g.Lxh;
  const uint32_t r1 = fdiv(r0, g.div_ly);
  c[1] = (int)(r0 - r1 * (uint32_t)g.L[1]);
  const uint32_t r2 = fdiv(r1, g.div_lz);
  c[2] = (int)(r1 - r2 * (uint32_t)g.L[2]);
  c[3] = (int)r2;
  c[0] = 2 * xh + ((p + c[1] + c[2] + c[3]) & 1);
}

// cb index and boundary phase of the neighbour of x (cb index i, coordinates c) in
// direction mu, forward (fwd = true) or backward.
__device__ __forceinline__ int cb_neighbour(const Geom& g, int i, const int c[4], int mu, bool fwd, int& phase) {
  phase = 1;
  if (mu == 0) {
    int xn;
    if (fwd) {
      xn = c[0] + 1;
      if (xn == g.L[0]) {
        xn = 0;
        phase = g.bc[0];
      }
    } else {
      xn = c[0] - 1;
      if (xn < 0) {
        xn = g.L[0] - 1;
        phase = g.bc[0];
      }
    }
    return i - (c[0] >> 1) + (xn >> 1);
  }
  const int L = g.L[mu];
  const int st = g.stride[mu];
  if (fwd) {
    if (c[mu] == L - 1) {
      phase = g.bc[mu];
      return i - (L - 1) * st;
    }
    return i + st;
  }
  if (c[mu] == 0) {
    phase = g.bc[mu];
    return i + (L - 1) * st;
  }
  return i - st;
}

}  // namespace gdwf
