// Site-local kernels: layout and precision conversion, standalone Mooee / Mooee^-1,
// FP64-accumulated reductions and CG vector updates. All are bandwidth-bound passes over the
// device field layout described in dwf_common.cuh.
//
// Elementwise kernels walk a field in units of 16 values: unit (site, g, q) is reals 8g..8g+7 of
// both slices of pair q of a site block, in the order [real][slice]. Consecutive threads take
// consecutive pairs, so every precision's 16-byte vectors are read and written contiguously, and
// fields of different precisions (whose vectors hold 1, 2 or 4 reals of two slices) can be
// combined in one pass. Pad slices (odd Ls) are zero and stay zero.
#include "dhop_kernel.cuh"
#include "site_ops.cuh"

namespace gdwf {

template <int P>
using RT = typename Store<P>::R;

template <int P>
__device__ __forceinline__ const char* site_ptr(const void* base, long site, int Lsh) {
  return static_cast<const char*>(base) + site_offset(site, Lsh, (size_t)Lsh * 2 * 24 * sizeof(typename Store<P>::T));
}

// The 16 values of unit (site, g, q): NV = 8 / RV vectors, chunks g*NV .. g*NV + NV - 1.
template <int P, bool COHERENT>
__device__ __forceinline__ void ld_unit(const void* base, long site, int g, int q, int Lsh, RT<P>* o) {
  constexpr int VEC = Store<P>::VEC;
  constexpr int NV = 16 / VEC;
  const char* sb = site_ptr<P>(base, site, Lsh);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const char* p = sb + (g * NV + v) * chunk_stride(Lsh) + (size_t)q * 16;
    if (COHERENT)
      ld16c<P>(p, o + v * VEC);
    else
      ld16<P>(p, o + v * VEC);
  }
}

template <int P>
__device__ __forceinline__ void st_unit(void* base, long site, int g, int q, int Lsh, const RT<P>* o) {
  constexpr int VEC = Store<P>::VEC;
  constexpr int NV = 16 / VEC;
  char* sb = const_cast<char*>(site_ptr<P>(base, site, Lsh));
#pragma unroll
  for (int v = 0; v < NV; ++v) st16<P>(sb + (g * NV + v) * chunk_stride(Lsh) + (size_t)q * 16, o + v * VEC);
}

template <int P>
__device__ __forceinline__ void st_unit_d(void* base, long site, int g, int q, int Lsh, const double* o) {
  constexpr int VEC = Store<P>::VEC;
  constexpr int NV = 16 / VEC;
  char* sb = const_cast<char*>(site_ptr<P>(base, site, Lsh));
#pragma unroll
  for (int v = 0; v < NV; ++v) st16d<P>(sb + (g * NV + v) * chunk_stride(Lsh) + (size_t)q * 16, o + v * VEC);
}

// Value i of a unit is real 8g + (i >> 1) of slice 2q + (i & 1).
__device__ __forceinline__ void unit_coords(long u, int Lsh, long& site, int& g, int& q) {
  const long rem = u / Lsh;
  q = (int)(u - rem * Lsh);
  site = rem / 3;
  g = (int)(rem - site * 3);
}

static inline int grid_for(long n, int threads) {
  long b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------- block reduction

template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double* partials, int nblocks) {
  __shared__ double red[N][RED_THREADS / 32];
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) red[k][warp] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double t = lane < RED_THREADS / 32 ? red[k][lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
      if (lane == 0) partials[k * nblocks + blockIdx.x] = t;
    }
  }
}

// Second pass: one CTA sums the RED_BLOCKS partials in a fixed order.
__global__ void __launch_bounds__(RED_THREADS) k_finalize(const double* partials, int ncomp, double* scal, int kind,
                                                         int dst) {
  __shared__ double red[2][RED_THREADS];
  for (int k = 0; k < ncomp; ++k) {
    double t = 0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += RED_THREADS) t += partials[k * RED_BLOCKS + i];
    red[k][threadIdx.x] = t;
  }
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < ncomp; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double tot = red[0][0];
    if (kind == FIN_STORE) {
      scal[dst] = tot;
      if (ncomp > 1) scal[dst + 1] = red[1][0];
    } else if (kind == FIN_ALPHA) {
      scal[S_PAP] = tot;
      scal[S_ALPHA] = scal[S_RR] / tot;
    } else if (kind == FIN_BETA) {
      scal[S_RRNEW] = tot;
      scal[S_BETA] = scal[S_PSCALE] * tot / scal[S_RR];
      scal[S_RROLD] = scal[S_RR];
      scal[S_RR] = tot;
      scal[S_PSCALE] = 1.0;
    }
  }
}

static cudaError_t finalize(const double* partials, int ncomp, double* scal, int kind, int dst, cudaStream_t st) {
  k_finalize<<<1, RED_THREADS, 0, st>>>(partials, ncomp, scal, kind, dst);
  return cudaGetLastError();
}

// n partials (any n) summed in a fixed order: thread t takes t, t + RED_THREADS, ..., then a tree.
__global__ void __launch_bounds__(RED_THREADS) k_finalize_n(const double* partials, int n, double* scal, int kind,
                                                           int dst) {
  __shared__ double red[RED_THREADS];
  double t = 0;
  for (int i = threadIdx.x; i < n; i += RED_THREADS) t += partials[i];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double tot = red[0];
    if (kind == FIN_STORE) {
      scal[dst] = tot;
    } else if (kind == FIN_ALPHA) {
      scal[S_PAP] = tot;
      scal[S_ALPHA] = scal[S_RR] / tot;
    } else if (kind == FIN_BETA) {
      scal[S_RRNEW] = tot;
      scal[S_BETA] = scal[S_PSCALE] * tot / scal[S_RR];
      scal[S_RROLD] = scal[S_RR];
      scal[S_RR] = tot;
      scal[S_PSCALE] = 1.0;
    }
  }
}

cudaError_t launch_finalize_n(const double* partials, int n, double* scal, int kind, int dst, cudaStream_t st) {
  k_finalize_n<<<1, RED_THREADS, 0, st>>>(partials, n, scal, kind, dst);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- pack / unpack

template <int P>
__global__ void k_pack_spinor(Geom g, double* canon, char* field, int parity0, int nparity, bool unpack) {
  using R = RT<P>;
  constexpr int VEC = Store<P>::VEC, RV = Store<P>::RV, NCH = Store<P>::NCH;
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const int Ls = g.Ls;
  const int Lsh = ls_half(Ls);
  const long total = (long)nparity * g.N4h * NCH * Lsh;
  if (tid >= total) return;
  const long rem = tid / Lsh;
  const int q = (int)(tid - rem * Lsh);
  const long sitep = rem / NCH;
  const int k = (int)(rem - sitep * NCH);
  const int ph = (int)(sitep / g.N4h);
  const int i = (int)(sitep - (long)ph * g.N4h);
  int c[4];
  cb_coords(g, i, parity0 + ph, c);
  const long lex = c[0] + (long)g.L[0] * (c[1] + (long)g.L[1] * (c[2] + (long)g.L[2] * c[3]));
  char* fp = field + site_offset(sitep, Lsh, (size_t)Lsh * 2 * 24 * sizeof(typename Store<P>::T)) + k * chunk_stride(Lsh) +
             (size_t)q * 16;
  // value 2j + l of the vector is real RV*k + j of slice 2q + l
  if (!unpack) {
    double v[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const int s = 2 * q + (e & 1);
      v[e] = s < Ls ? canon[(lex * Ls + s) * 24 + RV * k + (e >> 1)] : 0.0;
    }
    st16d<P>(fp, v);
  } else {
    R v[VEC];
    ld16<P>(fp, v);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const int s = 2 * q + (e & 1);
      if (s < Ls) canon[(lex * Ls + s) * 24 + RV * k + (e >> 1)] = (double)v[e];
    }
  }
}

cudaError_t launch_pack_spinor(int prec, const Geom& g, const double* canon, void* field, int subset, bool unpack,
                               cudaStream_t st) {
  const int parity0 = subset == 2 ? 0 : subset;
  const int nparity = subset == 2 ? 2 : 1;
  const long total = (long)nparity * g.N4h * (24 / (prec_vec(prec) / 2)) * ls_half(g.Ls);
  const int blocks = grid_for(total, 256);
  double* c = const_cast<double*>(canon);
  char* f = static_cast<char*>(field);
  switch (prec) {
    case P64: k_pack_spinor<P64><<<blocks, 256, 0, st>>>(g, c, f, parity0, nparity, unpack); break;
    case P32: k_pack_spinor<P32><<<blocks, 256, 0, st>>>(g, c, f, parity0, nparity, unpack); break;
    case P16: k_pack_spinor<P16><<<blocks, 256, 0, st>>>(g, c, f, parity0, nparity, unpack); break;
    default: k_pack_spinor<PB16><<<blocks, 256, 0, st>>>(g, c, f, parity0, nparity, unpack); break;
  }
  return cudaGetLastError();
}

template <int P, bool C12>
__global__ void k_pack_gauge(Geom g, const double* canon, char* Ue, char* Uo) {
  using R = RT<P>;
  constexpr int VEC = Store<P>::VEC;
  constexpr int LB = link_bytes(sizeof(typename Store<P>::T), C12);
  constexpr int NR = C12 ? 12 : 18;
  constexpr int NV = LB / 16;
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (tid >= 8L * g.N4h) return;
  const int mu = (int)(tid & 3);
  const long rem = tid >> 2;
  const int p = rem >= g.N4h ? 1 : 0;
  const int i = (int)(rem - (long)p * g.N4h);
  int c[4];
  cb_coords(g, i, p, c);
  const long lex = c[0] + (long)g.L[0] * (c[1] + (long)g.L[1] * (c[2] + (long)g.L[2] * c[3]));
  const double* u = canon + (lex * 4 + mu) * 18;
  char* dst = (p ? Uo : Ue) + ((size_t)i * 4 + mu) * LB;
  double buf[NV * VEC];
#pragma unroll
  for (int j = 0; j < NV * VEC; ++j) buf[j] = j < NR ? u[j] : 0.0;
#pragma unroll
  for (int v = 0; v < NV; ++v) st16d<P>(dst + v * 16, buf + v * VEC);
}

cudaError_t launch_pack_gauge(int prec, bool c12, const Geom& g, const double* canon, void* Ue, void* Uo,
                              cudaStream_t st) {
  const int blocks = grid_for(8L * g.N4h, 256);
  char* e = static_cast<char*>(Ue);
  char* o = static_cast<char*>(Uo);
#define PG(P_)                                                                   \
  if (c12)                                                                       \
    k_pack_gauge<P_, true><<<blocks, 256, 0, st>>>(g, canon, e, o);              \
  else                                                                           \
    k_pack_gauge<P_, false><<<blocks, 256, 0, st>>>(g, canon, e, o);
  switch (prec) {
    case P64: PG(P64) break;
    case P32: PG(P32) break;
    case P16: PG(P16) break;
    default: PG(PB16) break;
  }
#undef PG
  return cudaGetLastError();
}

// ---------------------------------------------------------------- precision conversion

template <int PS, int PD>
__global__ void k_convert(const void* src, void* dst, long nsites, int Ls, const double* scale_dev, double scale) {
  using RS = RT<PS>;
  using RD = RT<PD>;
  const double sc = scale_dev ? *scale_dev : scale;
  const int Lsh = ls_half(Ls);
  const long units = nsites * 3 * Lsh;
  for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < units; u += (long)gridDim.x * blockDim.x) {
    long site;
    int g, q;
    unit_coords(u, Lsh, site, g, q);
    RS a[16];
    ld_unit<PS, false>(src, site, g, q, Lsh, a);
    if constexpr (PS == P64 || PD == P64) {
      double b[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) b[j] = (double)a[j] * sc;
      st_unit_d<PD>(dst, site, g, q, Lsh, b);
    } else {
      RD b[16];
      const float f = (float)sc;
#pragma unroll
      for (int j = 0; j < 16; ++j) b[j] = (RD)((float)a[j] * f);
      st_unit<PD>(dst, site, g, q, Lsh, b);
    }
  }
}

cudaError_t launch_convert(int psrc, int pdst, const void* src, void* dst, long nsites, int Ls, const double* scale_dev,
                           double scale, cudaStream_t st) {
  const int blocks = grid_for(nsites * 3 * ls_half(Ls), 256);
#define CV(A, B) k_convert<A, B><<<blocks, 256, 0, st>>>(src, dst, nsites, Ls, scale_dev, scale)
#define CVROW(A)            \
  switch (pdst) {           \
    case P64: CV(A, P64); break;  \
    case P32: CV(A, P32); break;  \
    case P16: CV(A, P16); break;  \
    default: CV(A, PB16); break;  \
  }
  switch (psrc) {
    case P64: CVROW(P64) break;
    case P32: CVROW(P32) break;
    case P16: CVROW(P16) break;
    default: CVROW(PB16) break;
  }
#undef CVROW
#undef CV
  return cudaGetLastError();
}

// ---------------------------------------------------------------- standalone Mooee / Mooee^-1

// One CTA holds `spc` whole sites in shared memory (FP32 or FP64 arithmetic): load, apply the
// fifth-dimension operator, store. in and out may be the same buffer.
template <int P>
__global__ void __launch_bounds__(256) k_mooee(const void* in, void* out, long nsites, int Ls, int spc, bool dag,
                                               bool inverse, double d5, double mass, double inv_d5, double inv_den) {
  using R = RT<P>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);  // [site][s < Ls][24 reals, padded to INV_SLICE_STRIDE]
  constexpr int S = INV_SLICE_STRIDE;
  const int Lsh = ls_half(Ls);
  const long site0 = (long)blockIdx.x * spc;
  const int ns = (int)min((long)spc, nsites - site0);
  const int units = ns * 3 * Lsh;
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    const int rem = u / Lsh;
    const int q = u - rem * Lsh;
    const int sl = rem / 3;
    const int g = rem - sl * 3;
    R v[16];
    ld_unit<P, true>(in, site0 + sl, g, q, Lsh, v);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int s = 2 * q + (i & 1);
      if (s < Ls) sm[((size_t)sl * Ls + s) * S + 8 * g + (i >> 1)] = v[i];
    }
  }
  __syncthreads();
  if (inverse) {
    for (int task = threadIdx.x; task < ns * 24; task += blockDim.x) {
      const int sl = task / 24;
      const int r = task - sl * 24;
      const bool upper = r < 12;
      mooee_inv_line<R>(sm + (size_t)sl * Ls * S + r, Ls, dag ? !upper : upper, R(mass), R(inv_d5), R(inv_den));
    }
    __syncthreads();
    for (int u = threadIdx.x; u < units; u += blockDim.x) {
      const int rem = u / Lsh;
      const int q = u - rem * Lsh;
      const int sl = rem / 3;
      const int g = rem - sl * 3;
      R o[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int s = 2 * q + (i & 1);
        o[i] = s < Ls ? sm[((size_t)sl * Ls + s) * S + 8 * g + (i >> 1)] : R(0);
      }
      st_unit<P>(out, site0 + sl, g, q, Lsh, o);
    }
    return;
  }
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    const int rem = u / Lsh;
    const int q = u - rem * Lsh;
    const int sl = rem / 3;
    const int g = rem - sl * 3;
    const R* base = sm + (size_t)sl * Ls * S;
    R o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int s = 2 * q + (i & 1);
      const int r = 8 * g + (i >> 1);
      if (s >= Ls) {
        o[i] = R(0);
        continue;
      }
      const int sm1 = s > 0 ? s - 1 : Ls - 1, sp1 = s < Ls - 1 ? s + 1 : 0;
      const R cm = s > 0 ? R(-1) : R(mass), cp = s < Ls - 1 ? R(-1) : R(mass);
      const int s_up = dag ? sp1 : sm1, s_lo = dag ? sm1 : sp1;
      const R c_up = dag ? cp : cm, c_lo = dag ? cm : cp;
      const bool upper = r < 12;
      o[i] = R(d5) * base[s * S + r] + (upper ? c_up * base[s_up * S + r] : c_lo * base[s_lo * S + r]);
    }
    st_unit<P>(out, site0 + sl, g, q, Lsh, o);
  }
}

cudaError_t launch_mooee(int prec, const void* in, void* out, long nsites, int Ls, bool dag, bool inverse, double d5,
                         double mass, double inv_d5, double inv_den, cudaStream_t st) {
  const size_t rbytes = prec == P64 ? 8 : 4;
  const size_t site_smem = (size_t)Ls * INV_SLICE_STRIDE * rbytes;
  int spc = (int)((48 * 1024) / site_smem);
  if (spc > 64) spc = 64;
  if (spc < 1) return cudaErrorInvalidValue;
  const size_t smem = spc * site_smem;
  const int blocks = grid_for(nsites, spc);
#define MO(P_) k_mooee<P_><<<blocks, 256, smem, st>>>(in, out, nsites, Ls, spc, dag, inverse, d5, mass, inv_d5, inv_den)
  switch (prec) {
    case P64: MO(P64); break;
    case P32: MO(P32); break;
    case P16: MO(P16); break;
    default: MO(PB16); break;
  }
#undef MO
  return cudaGetLastError();
}

// ---------------------------------------------------------------- reductions

// Sum over 8 reals of a unit: |a|^2, or the complex a^+ b. Lower precisions form the 8-term
// partial in FP32 and add it to the FP64 accumulator; FP64 data is accumulated in FP64.
template <int P, bool INNER>
__global__ void __launch_bounds__(RED_THREADS) k_reduce(const void* a, const void* b, long nsites, int Ls,
                                                        double* partials) {
  using R = RT<P>;
  double acc[2] = {0.0, 0.0};
  const int Lsh = ls_half(Ls);
  const long units = nsites * 3 * Lsh;
  for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < units; u += (long)gridDim.x * blockDim.x) {
    long site;
    int g, q;
    unit_coords(u, Lsh, site, g, q);
    R x[16];
    ld_unit<P, false>(a, site, g, q, Lsh, x);
    if (INNER) {
      R y[16];
      ld_unit<P, false>(b, site, g, q, Lsh, y);
      R re = 0, im = 0;
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          const int ir = (2 * c) * 2 + l, ii = (2 * c + 1) * 2 + l;  // re and im of one complex number
          re += x[ir] * y[ir] + x[ii] * y[ii];
          im += x[ir] * y[ii] - x[ii] * y[ir];
        }
      acc[0] += (double)re;
      acc[1] += (double)im;
    } else {
      R t = 0;
#pragma unroll
      for (int j = 0; j < 16; ++j) t += x[j] * x[j];
      acc[0] += (double)t;
    }
  }
  if (INNER) {
    block_sum<2>(acc, partials, RED_BLOCKS);
  } else {
    double v[1] = {acc[0]};
    block_sum<1>(v, partials, RED_BLOCKS);
  }
}

cudaError_t launch_reduce(int prec, const void* a, const void* b, long nsites, int Ls, double* partials, double* scal,
                          int kind, int dst, cudaStream_t st) {
  const bool inner = b != nullptr;
#define RD(P_)                                                                              \
  if (inner)                                                                                \
    k_reduce<P_, true><<<RED_BLOCKS, RED_THREADS, 0, st>>>(a, b, nsites, Ls, partials);     \
  else                                                                                      \
    k_reduce<P_, false><<<RED_BLOCKS, RED_THREADS, 0, st>>>(a, b, nsites, Ls, partials);
  switch (prec) {
    case P64: RD(P64) break;
    case P32: RD(P32) break;
    case P16: RD(P16) break;
    default: RD(PB16) break;
  }
#undef RD
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return finalize(partials, inner ? 2 : 1, scal, kind, dst, st);
}

// ---------------------------------------------------------------- CG updates

template <int PX, int PP>
__global__ void __launch_bounds__(RED_THREADS) k_cg_xr(void* x, void* r, const void* p, const void* Ap, long nsites,
                                                       int Ls, const double* scal, double* partials) {
  using RX = RT<PX>;
  using RP = RT<PP>;
  const RX alpha = (RX)scal[S_ALPHA];
  double acc = 0.0;
  const int Lsh = ls_half(Ls);
  const long units = nsites * 3 * Lsh;
  for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < units; u += (long)gridDim.x * blockDim.x) {
    long site;
    int g, q;
    unit_coords(u, Lsh, site, g, q);
    RX xv[16], rv[16];
    RP pv[16], av[16];
    ld_unit<PX, true>(x, site, g, q, Lsh, xv);
    ld_unit<PX, true>(r, site, g, q, Lsh, rv);
    ld_unit<PP, false>(p, site, g, q, Lsh, pv);
    ld_unit<PP, false>(Ap, site, g, q, Lsh, av);
    RX t = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      xv[j] += alpha * (RX)pv[j];
      rv[j] -= alpha * (RX)av[j];
      t += rv[j] * rv[j];
    }
    st_unit<PX>(x, site, g, q, Lsh, xv);
    st_unit<PX>(r, site, g, q, Lsh, rv);
    acc += (double)t;
  }
  double v[1] = {acc};
  block_sum<1>(v, partials, RED_BLOCKS);
}

template <int PX, int PP>
__global__ void k_cg_p(const void* r, void* p, long nsites, int Ls, const double* scal) {
  using RX = RT<PX>;
  using RP = RT<PP>;
  const RX beta = (RX)scal[S_BETA];
  const int Lsh = ls_half(Ls);
  const long units = nsites * 3 * Lsh;
  for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < units; u += (long)gridDim.x * blockDim.x) {
    long site;
    int g, q;
    unit_coords(u, Lsh, site, g, q);
    RX rv[16];
    RP pv[16];
    ld_unit<PX, false>(r, site, g, q, Lsh, rv);
    ld_unit<PP, true>(p, site, g, q, Lsh, pv);
#pragma unroll
    for (int j = 0; j < 16; ++j) pv[j] = (RP)(rv[j] + beta * (RX)pv[j]);
    st_unit<PP>(p, site, g, q, Lsh, pv);
  }
}

// The mixed solver's inner loop, with the x update deferred by one pass so that p is read once
// per iteration: k_cg_r forms r -= alpha Ap and |r|^2 (reads r, Ap), then k_cg_xp forms
// x += alpha p and p = r + beta p from the same read of p (reads x, r, p). Ten field passes per
// iteration (with p^+ Ap) instead of eleven. k_cg_x applies the pending x update alone, before a
// reliable update folds x into the FP64 solution.
template <int PX, int PP>
__global__ void __launch_bounds__(RED_THREADS) k_cg_r(void* r, const void* Ap, long nsites, int Ls, const double* scal,
                                                      double* partials) {
  using RX = RT<PX>;
  using RP = RT<PP>;
  const RX alpha = (RX)scal[S_ALPHA];
  double acc = 0.0;
  const int Lsh = ls_half(Ls);
  const long units = nsites * 3 * Lsh;
  for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < units; u += (long)gridDim.x * blockDim.x) {
    long site;
    int g, q;
    unit_coords(u, Lsh, site, g, q);
    RX rv[16];
    RP av[16];
    ld_unit<PX, true>(r, site, g, q, Lsh, rv);
    ld_unit<PP, false>(Ap, site, g, q, Lsh, av);
    RX t = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      rv[j] -= alpha * (RX)av[j];
      t += rv[j] * rv[j];
    }
    st_unit<PX>(r, site, g, q, Lsh, rv);
    acc += (double)t;
  }
  double v[1] = {acc};
  block_sum<1>(v, partials, RED_BLOCKS);
}

template <int PX, int PP, bool UPDATE_P>
__global__ void k_cg_xp(void* x, const void* r, void* p, long nsites, int Ls, const double* scal) {
  using RX = RT<PX>;
  using RP = RT<PP>;
  const RX alpha = (RX)scal[S_ALPHA];
  const RX beta = (RX)scal[S_BETA];
  const int Lsh = ls_half(Ls);
  const long units = nsites * 3 * Lsh;
  for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < units; u += (long)gridDim.x * blockDim.x) {
    long site;
    int g, q;
    unit_coords(u, Lsh, site, g, q);
    RX xv[16], rv[16];
    RP pv[16];
    ld_unit<PX, true>(x, site, g, q, Lsh, xv);
    ld_unit<PP, UPDATE_P>(p, site, g, q, Lsh, pv);  // coherent when p is rewritten
    if (UPDATE_P) ld_unit<PX, false>(r, site, g, q, Lsh, rv);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      xv[j] += alpha * (RX)pv[j];
      if (UPDATE_P) pv[j] = (RP)(rv[j] + beta * (RX)pv[j]);
    }
    st_unit<PX>(x, site, g, q, Lsh, xv);
    if (UPDATE_P) st_unit<PP>(p, site, g, q, Lsh, pv);
  }
}

#define CG_PAIRS(M) \
  M(P64, P64)       \
  M(P32, P32)       \
  M(P32, P16)       \
  M(P32, PB16)

cudaError_t launch_cg_xr(int px, int pp, void* x, void* r, const void* p, const void* Ap, long nsites, int Ls,
                         double* partials, double* scal, cudaStream_t st) {
#define XR(A, B)                                                                                  \
  if (px == A && pp == B) {                                                                       \
    k_cg_xr<A, B><<<RED_BLOCKS, RED_THREADS, 0, st>>>(x, r, p, Ap, nsites, Ls, scal, partials);  \
    cudaError_t e = cudaGetLastError();                                                           \
    if (e != cudaSuccess) return e;                                                               \
    return finalize(partials, 1, scal, FIN_BETA, 0, st);                                          \
  }
  CG_PAIRS(XR)
#undef XR
  return cudaErrorInvalidValue;
}

cudaError_t launch_cg_r(int px, int pp, void* r, const void* Ap, long nsites, int Ls, double* partials, double* scal,
                        cudaStream_t st) {
#define RU(A, B)                                                                             \
  if (px == A && pp == B) {                                                                  \
    k_cg_r<A, B><<<RED_BLOCKS, RED_THREADS, 0, st>>>(r, Ap, nsites, Ls, scal, partials);    \
    cudaError_t e = cudaGetLastError();                                                      \
    if (e != cudaSuccess) return e;                                                          \
    return finalize(partials, 1, scal, FIN_BETA, 0, st);                                     \
  }
  CG_PAIRS(RU)
#undef RU
  return cudaErrorInvalidValue;
}

cudaError_t launch_cg_xp(int px, int pp, void* x, const void* r, void* p, long nsites, int Ls, const double* scal,
                         bool update_p, cudaStream_t st) {
  const int blocks = grid_for(nsites * 3 * ls_half(Ls), 256);
#define XP(A, B)                                                                                        \
  if (px == A && pp == B) {                                                                             \
    if (update_p)                                                                                       \
      k_cg_xp<A, B, true><<<blocks, 256, 0, st>>>(x, r, p, nsites, Ls, scal);                          \
    else                                                                                                \
      k_cg_xp<A, B, false><<<blocks, 256, 0, st>>>(x, r, p, nsites, Ls, scal);                         \
    return cudaGetLastError();                                                                          \
  }
  CG_PAIRS(XP)
#undef XP
  return cudaErrorInvalidValue;
}

cudaError_t launch_cg_p(int px, int pp, const void* r, void* p, long nsites, int Ls, const double* scal,
                        cudaStream_t st) {
  const int blocks = grid_for(nsites * 3 * ls_half(Ls), 256);
#define PU(A, B)                                                              \
  if (px == A && pp == B) {                                                   \
    k_cg_p<A, B><<<blocks, 256, 0, st>>>(r, p, nsites, Ls, scal);             \
    return cudaGetLastError();                                                \
  }
  CG_PAIRS(PU)
#undef PU
  return cudaErrorInvalidValue;
}

__global__ void __launch_bounds__(RED_THREADS) k_residual64(const void* b, const void* Ax, void* r, long nsites, int Ls,
                                                            double* partials) {
  double acc = 0.0;
  const int Lsh = ls_half(Ls);
  const long units = nsites * 3 * Lsh;
  for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < units; u += (long)gridDim.x * blockDim.x) {
    long site;
    int g, q;
    unit_coords(u, Lsh, site, g, q);
    double bv[16], av[16];
    ld_unit<P64, false>(b, site, g, q, Lsh, bv);
    ld_unit<P64, false>(Ax, site, g, q, Lsh, av);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      bv[j] -= av[j];
      acc += bv[j] * bv[j];
    }
    st_unit<P64>(r, site, g, q, Lsh, bv);
  }
  double v[1] = {acc};
  block_sum<1>(v, partials, RED_BLOCKS);
}

cudaError_t launch_residual64(const void* b, const void* Ax, void* r, long nsites, int Ls, double* partials,
                              double* scal, int dst, cudaStream_t st) {
  k_residual64<<<RED_BLOCKS, RED_THREADS, 0, st>>>(b, Ax, r, nsites, Ls, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return finalize(partials, 1, scal, FIN_STORE, dst, st);
}

template <int PY>
__global__ void k_accum_zero(void* x, void* y, long nsites, int Ls, const double* c_dev) {
  using RY = RT<PY>;
  const double c = *c_dev;
  const int Lsh = ls_half(Ls);
  const long units = nsites * 3 * Lsh;
  for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < units; u += (long)gridDim.x * blockDim.x) {
    long site;
    int g, q;
    unit_coords(u, Lsh, site, g, q);
    double xv[16];
    RY yv[16];
    ld_unit<P64, true>(x, site, g, q, Lsh, xv);
    ld_unit<PY, true>(y, site, g, q, Lsh, yv);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      xv[j] += c * (double)yv[j];
      yv[j] = RY(0);
    }
    st_unit<P64>(x, site, g, q, Lsh, xv);
    st_unit<PY>(y, site, g, q, Lsh, yv);
  }
}

cudaError_t launch_accum_zero(int py, void* x, void* y, long nsites, int Ls, const double* c_dev, cudaStream_t st) {
  const int blocks = grid_for(nsites * 3 * ls_half(Ls), 256);
  switch (py) {
    case P64: k_accum_zero<P64><<<blocks, 256, 0, st>>>(x, y, nsites, Ls, c_dev); break;
    case P32: k_accum_zero<P32><<<blocks, 256, 0, st>>>(x, y, nsites, Ls, c_dev); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int P>
__global__ void k_axpby(double a, const void* x, double b, void* y, long nsites, int Ls) {
  using R = RT<P>;
  const int Lsh = ls_half(Ls);
  const long units = nsites * 3 * Lsh;
  for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < units; u += (long)gridDim.x * blockDim.x) {
    long site;
    int g, q;
    unit_coords(u, Lsh, site, g, q);
    R xv[16], yv[16];
    ld_unit<P, true>(x, site, g, q, Lsh, xv);
    ld_unit<P, true>(y, site, g, q, Lsh, yv);
#pragma unroll
    for (int j = 0; j < 16; ++j) yv[j] = R(a) * xv[j] + R(b) * yv[j];
    st_unit<P>(y, site, g, q, Lsh, yv);
  }
}

cudaError_t launch_axpby(int p, double a, const void* x, double b, void* y, long nsites, int Ls, cudaStream_t st) {
  const int blocks = grid_for(nsites * 3 * ls_half(Ls), 256);
  switch (p) {
    case P64: k_axpby<P64><<<blocks, 256, 0, st>>>(a, x, b, y, nsites, Ls); break;
    case P32: k_axpby<P32><<<blocks, 256, 0, st>>>(a, x, b, y, nsites, Ls); break;
    case P16: k_axpby<P16><<<blocks, 256, 0, st>>>(a, x, b, y, nsites, Ls); break;
    default: k_axpby<PB16><<<blocks, 256, 0, st>>>(a, x, b, y, nsites, Ls); break;
  }
  return cudaGetLastError();
}

}  // namespace gdwf

// ---------------------------------------------------------------- reduction without allocation
//
// grid_dwf_inner_noalloc: the same FP64-accumulated reduction as launch_reduce, for callers
// that must not allocate device memory, with its scratch in a fixed array that is part of the
// library's device image instead of a cudaMalloc'd buffer. Each CTA reduces one contiguous
// chunk of NOALLOC_UNITS_PER_CTA units (16 values each), so the number of partial sums, and with
// it the largest field accepted, is bounded by the array.

namespace gdwf {

constexpr int NOALLOC_UNITS_PER_THREAD = 8;
constexpr long NOALLOC_UNITS_PER_CTA = (long)RED_THREADS * NOALLOC_UNITS_PER_THREAD;
constexpr int NOALLOC_MAX_PARTIALS = 16384;
constexpr int NOALLOC_MAX_DEVICES = 64;

// [re partials][im partials]: 256 KiB on every device that loads the library, held until the
// process exits.
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_PARTIALS];

template <int P, bool INNER>
__global__ void __launch_bounds__(RED_THREADS) k_reduce_chunked(const void* a, const void* b, long nsites, int Ls,
                                                                double* partials, int nblocks) {
  using R = RT<P>;
  double acc[2] = {0.0, 0.0};
  const int Lsh = ls_half(Ls);
  const long units = nsites * 3 * Lsh;
  const long first = (long)blockIdx.x * NOALLOC_UNITS_PER_CTA;
#pragma unroll
  for (int k = 0; k < NOALLOC_UNITS_PER_THREAD; ++k) {
    const long u = first + threadIdx.x + (long)k * RED_THREADS;
    if (u >= units) break;
    long site;
    int g, q;
    unit_coords(u, Lsh, site, g, q);
    R x[16];
    ld_unit<P, false>(a, site, g, q, Lsh, x);
    if (INNER) {
      R y[16];
      ld_unit<P, false>(b, site, g, q, Lsh, y);
      R re = 0, im = 0;
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          const int ir = (2 * c) * 2 + l, ii = (2 * c + 1) * 2 + l;  // re and im of one complex number
          re += x[ir] * y[ir] + x[ii] * y[ii];
          im += x[ir] * y[ii] - x[ii] * y[ir];
        }
      acc[0] += (double)re;
      acc[1] += (double)im;
    } else {
      R t = 0;
#pragma unroll
      for (int j = 0; j < 16; ++j) t += x[j] * x[j];
      acc[0] += (double)t;
    }
  }
  block_sum<2>(acc, partials, nblocks);
}

// One CTA adds the nblocks partials in a fixed order and writes (re, im) to out.
__global__ void __launch_bounds__(RED_THREADS) k_finalize_chunked(const double* partials, int nblocks, double* out) {
  __shared__ double red[2][RED_THREADS];
  for (int k = 0; k < 2; ++k) {
    double t = 0;
    for (int i = threadIdx.x; i < nblocks; i += RED_THREADS) t += partials[k * nblocks + i];
    red[k][threadIdx.x] = t;
  }
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 2; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = red[0][0];
    out[1] = red[1][0];
  }
}

}  // namespace gdwf

#include <mutex>
#include <string>

#include "../../include/grid_dwf.h"

namespace {

double* g_noalloc_dev_ptr[gdwf::NOALLOC_MAX_DEVICES] = {};
std::mutex g_noalloc_mutex;

int noalloc_error(char* err, size_t err_len, int code, const std::string& msg) {
  if (err && err_len > 0) {
    const size_t n = msg.size() < err_len - 1 ? msg.size() : err_len - 1;
    memcpy(err, msg.data(), n);
    err[n] = '\0';
  }
  return code;
}

}  // namespace

extern "C" int grid_dwf_inner_noalloc(int precision, const void* a, const void* b, long nsites, int Ls, void* stream,
                                      double* result, char* err, size_t err_len) {
  using namespace gdwf;
  if (err && err_len > 0) err[0] = '\0';
  if (precision < GRID_DWF_FP64 || precision > GRID_DWF_BF16)
    return noalloc_error(err, err_len, GRID_DWF_ERR_INVALID_ARG, "grid_dwf_inner_noalloc: bad precision");
  if (!a || !result || nsites < 0 || Ls < 1)
    return noalloc_error(err, err_len, GRID_DWF_ERR_INVALID_ARG, "grid_dwf_inner_noalloc: null pointer or bad size");
  // Sites are stored in blocks of SITE_BLOCK: a partial last block would make the kernel read the
  // chunks of a whole block past the end of a buffer sized for nsites sites.
  if (nsites % SITE_BLOCK != 0)
    return noalloc_error(err, err_len, GRID_DWF_ERR_INVALID_ARG,
                         "grid_dwf_inner_noalloc: nsites must be a multiple of " + std::to_string(SITE_BLOCK) +
                             " (fields hold whole blocks of 4 checkerboard sites)");
  if (reinterpret_cast<uintptr_t>(a) % 16 || (b && reinterpret_cast<uintptr_t>(b) % 16) ||
      reinterpret_cast<uintptr_t>(result) % 8)
    return noalloc_error(err, err_len, GRID_DWF_ERR_INVALID_ARG, "grid_dwf_inner_noalloc: misaligned pointer");
  const long Lsh = ls_half(Ls);
  const long units = nsites * 3L * Lsh;  // 16 values (8 reals of a slice pair) each
  const long nblocks = (units + NOALLOC_UNITS_PER_CTA - 1) / NOALLOC_UNITS_PER_CTA;
  if (nsites > 0 && (units / 3 / Lsh != nsites || nblocks > NOALLOC_MAX_PARTIALS))
    return noalloc_error(err, err_len, GRID_DWF_ERR_INVALID_ARG,
                         "grid_dwf_inner_noalloc: field of " + std::to_string(nsites) + " sites x Ls " +
                             std::to_string(Ls) + " exceeds the static scratch (at most " +
                             std::to_string((long)NOALLOC_MAX_PARTIALS * NOALLOC_UNITS_PER_CTA / 3 * 2) +
                             " five-dimensional sites, nsites * Ls rounded up to even)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return noalloc_error(err, err_len, GRID_DWF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
    return noalloc_error(err, err_len, GRID_DWF_ERR_INVALID_ARG, "grid_dwf_inner_noalloc: device index too large");
  double* scratch = nullptr;
  {
    // Set-up, once per device, with that device current: the device address of the array.
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_dev_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return noalloc_error(err, err_len, GRID_DWF_ERR_CUDA,
                             std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_noalloc_dev_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_noalloc_dev_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nb = nblocks > 0 ? (int)nblocks : 1;
  const bool inner = b != nullptr;
#define NA(P_)                                                                                         \
  if (inner)                                                                                           \
    k_reduce_chunked<P_, true><<<nb, RED_THREADS, 0, st>>>(a, b, nsites, Ls, scratch, nb);             \
  else                                                                                                 \
    k_reduce_chunked<P_, false><<<nb, RED_THREADS, 0, st>>>(a, b, nsites, Ls, scratch, nb);
  switch (precision) {
    case P64: NA(P64) break;
    case P32: NA(P32) break;
    case P16: NA(P16) break;
    default: NA(PB16) break;
  }
#undef NA
  k_finalize_chunked<<<1, RED_THREADS, 0, st>>>(scratch, nb, result);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return noalloc_error(err, err_len, GRID_DWF_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return GRID_DWF_OK;
}
