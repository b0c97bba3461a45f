// The FP64 hopping stencil in float-float arithmetic: FP64 fields and links in memory, every
// real carried in registers as an unevaluated sum hi + lo of two FP32 numbers.
//
// Why. On this part the FP64 pipe retires about two fused multiply-adds per SM and clock,
// against 128 FP32 ones, so the FP64 kernel of dhop_kernel.cuh is bound by that pipe: it needs
// about 20 times longer for its arithmetic than HBM needs for its bytes. A float-float operation
// costs between 2 and 12 FP32 instructions, so the same operator in float-float runs on the wide
// FP32 pipe instead. The format is Dekker's double-length arithmetic ("A floating-point technique
// for extending the available precision", Numer. Math. 18, 1971): a sum is formed with Knuth's
// error-free TwoSum, a product with the FMA-based TwoProduct (the rounding error of a*b is
// fma(a, b, -a*b) exactly). A value carries about 47 significant bits (2^-47 ~ 7e-15 relative),
// enough for parity with the FP64 operator at 1e-12 and for the FP64 true residuals of the
// solvers; its exponent range is FP32's, so magnitudes below 2^-103 (~1e-31) are flushed to zero
// and above 2^128 become infinite.
//
// Same operator, layout, thread mapping (one thread per (site, slice)), link staging and fused
// epilogues (out = post(alpha Dhop in + beta pre(aux))) as the FP64 kernel; see there.
#include "dhop_ff.cuh"
#include "ff_arith.cuh"

namespace gdwf {
namespace {

using namespace ffa;

// ---------------------------------------------------------------- the hop loop's code shape
// The loops over hops and colour rows below are not unrolled: unrolled, the float-float
// arithmetic of eight hops is about 300 KB of machine code, far more than the SM's instruction
// caches, and the warps stalled on instruction fetch. So every hop runs the same short code: the
// lower spins of the projection are loaded at hop-dependent addresses with their signs flipped on
// load (the projection's additions run in FP64: the stored reals are FP64 anyway); the link is
// staged as U or U^+ so that the colour product has one form; the product is written to a
// per-thread shared-memory slot, from which the reconstruction of the lower spins reads at
// hop-dependent addresses.

// Row a of o = U h for both spins: u the row's 3 complex entries (6 ff), h the half spinor.
// Each output real is a six-term dot product, returned as its unnormalised pair (S, E).
__device__ __forceinline__ void su3_row_ff(const ff* u, const ff* h, ff* o /* [sp][re, im] */) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    ffacc re, im;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const ff ur = u[b * 2], ui = u[b * 2 + 1];
      const ff hr = h[(sp * 3 + b) * 2], hi = h[(sp * 3 + b) * 2 + 1];
      // re += ur hr - ui hi, im += ur hi + ui hr
      if (b == 0) {
        dot_first(re, ur, hr, false);
        dot_first(im, ur, hi, false);
      } else {
        dot_add<+1>(re, ur, hr);
        dot_add<+1>(im, ur, hi);
      }
      dot_add<-1>(re, ui, hi);
      dot_add<+1>(im, ui, hr);
    }
    o[sp * 2] = ff_make(re.s, re.e);  // unnormalised: only ever added into an accumulator
    o[sp * 2 + 1] = ff_make(im.s, im.e);
  }
}

// ---------------------------------------------------------------- memory

// The 24 reals of slice s of a site block (FP64 layout: real k at k * chunk_stride + s * 8).
template <int LSH>
__device__ __forceinline__ void load_slice_ff(const char* blk, int s, int Lsh_rt, ff* v) {
  const int Lsh = LSH > 0 ? LSH : Lsh_rt;
  const char* b = blk + (size_t)s * 8;
  double d[24];
#pragma unroll
  for (int k = 0; k < 24; ++k) d[k] = __ldg(reinterpret_cast<const double*>(b + k * chunk_stride(Lsh)));
#pragma unroll
  for (int k = 0; k < 24; ++k) v[k] = ff_from_double(d[k]);
}

// Reals r0 .. r0 + 11 of slice s.
template <int LSH>
__device__ __forceinline__ void load_half_ff(const char* blk, int s, int Lsh_rt, int r0, ff* v) {
  const int Lsh = LSH > 0 ? LSH : Lsh_rt;
  const char* b = blk + (size_t)s * 8;
  double d[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) d[k] = __ldg(reinterpret_cast<const double*>(b + (r0 + k) * chunk_stride(Lsh)));
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = ff_from_double(d[k]);
}

template <int LSH>
__device__ __forceinline__ void store_slice_ff(char* blk, int s, int Lsh_rt, const ff* v) {
  const int Lsh = LSH > 0 ? LSH : Lsh_rt;
  char* b = blk + (size_t)s * 8;
#pragma unroll
  for (int k = 0; k < 24; ++k) *reinterpret_cast<double*>(b + k * chunk_stride(Lsh)) = ff_to_double(v[k]);
}

template <int LSH>
__device__ __forceinline__ void store_zero_slice(char* blk, int s, int Lsh_rt) {
  const int Lsh = LSH > 0 ? LSH : Lsh_rt;
  char* b = blk + (size_t)s * 8;
#pragma unroll
  for (int k = 0; k < 24; ++k) *reinterpret_cast<double*>(b + k * chunk_stride(Lsh)) = 0.0;
}

// One stored FP64 link (18 or 12 reals) times the boundary phase, as the 18 ff of U (forward hop)
// or of U^+ (backward hop) in shared memory.
template <bool C12>
__device__ __forceinline__ void stage_link_ff(ff* dst, const char* src, bool negate, bool adjoint) {
  double u[18];
  load_link<P64, C12>(src, u);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      // both candidates at compile-time indices (a runtime index would put u in local memory)
      ff re = ff_from_double(adjoint ? u[(b * 3 + a) * 2] : u[(a * 3 + b) * 2]);
      ff im = ff_from_double(adjoint ? u[(b * 3 + a) * 2 + 1] : u[(a * 3 + b) * 2 + 1]);
      if (negate) re = ff_neg(re);
      if (negate != adjoint) im = ff_neg(im);
      dst[(a * 3 + b) * 2] = re;
      dst[(a * 3 + b) * 2 + 1] = im;
    }
}

// In-place inverse of the fifth-dimension matrix along one real of one site (stride INV_SLICE_STRIDE
// between slices), the float-float form of mooee_inv_line.
__device__ __forceinline__ void mooee_inv_line_ff(ff* v, int Ls, bool forward_form, ff mass, ff inv_d, ff inv_den) {
  if (forward_form) {
    ff acc = ff_make(0.f, 0.f);
    for (int k = 1; k < Ls; ++k) acc = ff_mul(ff_add<+1>(acc, v[k * INV_SLICE_STRIDE]), inv_d);
    ff y = ff_mul(ff_add<-1>(v[0], ff_mul(mass, acc)), inv_den);
    v[0] = y;
    for (int s = 1; s < Ls; ++s) {
      y = ff_mul(ff_add<+1>(v[s * INV_SLICE_STRIDE], y), inv_d);
      v[s * INV_SLICE_STRIDE] = y;
    }
  } else {
    ff acc = ff_make(0.f, 0.f);
    for (int k = Ls - 2; k >= 0; --k) acc = ff_mul(ff_add<+1>(acc, v[k * INV_SLICE_STRIDE]), inv_d);
    ff y = ff_mul(ff_add<-1>(v[(Ls - 1) * INV_SLICE_STRIDE], ff_mul(mass, acc)), inv_den);
    v[(Ls - 1) * INV_SLICE_STRIDE] = y;
    for (int s = Ls - 2; s >= 0; --s) {
      y = ff_mul(ff_add<+1>(v[s * INV_SLICE_STRIDE], y), inv_d);
      v[s * INV_SLICE_STRIDE] = y;
    }
  }
}

// ---------------------------------------------------------------- kernel

constexpr int FF_LINK_SITE_BYTES = 8 * 18 * 8;
constexpr int FF_UH_BYTES = 12 * 128 * 8;  // colour-product slots of up to 128 threads

// Four CTAs of 128 threads per SM (128 registers per thread; measured 2% faster than three CTAs
// with 168 registers).
#ifndef DWF_FF_MIN_BLOCKS
#define DWF_FF_MIN_BLOCKS 4
#endif

template <bool DAG, bool C12, int LSC>
__global__ void __launch_bounds__(128, DWF_FF_MIN_BLOCKS) dhop_kernel_ff(const __grid_constant__ DhopArgs a) {
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
  const size_t cs = chunk_stride(Lsh);

  // shared memory: [site][hop 8][18 ff] links, [site][hop 8] neighbour indices, [real 12][thread]
  // colour products (ff), then (post-operation) [site][Ls][24 ff]
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ff* lsm = reinterpret_cast<ff*>(smem_raw) + (size_t)site_local * 8 * 18;
  int* nbs = reinterpret_cast<int*>(smem_raw + (size_t)a.sites_per_cta * FF_LINK_SITE_BYTES) + site_local * 8;
  if (active) {
    int c[4];
    cb_coords(a.g, site, a.out_parity, c);
    const char* Uo = static_cast<const char*>(a.Uout);
    const char* Ui = static_cast<const char*>(a.Uin);
    // thread s stages the links of hops s, s + Lsp, ... and records their neighbour sites
    for (int h = s; h < 8; h += Lsp) {
      const int mu = h >> 1;
      const bool fwd = (h & 1) == 0;
      int ph;
      const int nb = cb_neighbour(a.g, site, c, mu, fwd, ph);
      const char* src = fwd ? Uo + ((size_t)site * 4 + mu) * LB : Ui + ((size_t)nb * 4 + mu) * LB;
      stage_link_ff<C12>(lsm + h * 18, src, ph < 0, !fwd);
      nbs[h] = nb;
    }
  }
  __syncthreads();

  ff acc[24];
#pragma unroll
  for (int r = 0; r < 24; ++r) acc[r] = ff_make(0.f, 0.f);
  if (active) {
    const char* in = static_cast<const char*>(a.in) + (size_t)s * 8;
    const int bd = blockDim.x;
    ff* uhs = reinterpret_cast<ff*>(smem_raw + (size_t)a.sites_per_cta * (FF_LINK_SITE_BYTES + 32)) + tid;
#pragma unroll 1
    for (int hop = 0; hop < 8; ++hop) {
      const int mu = hop >> 1;
      const int S = (hop & 1) == 0 ? SF : SB;
      const char* blk = in + site_offset(nbs[hop], Lsh, site_bytes);
      ff h[12];
      project_load_ff(blk, mu, S, cs, h);
      // uh = U h (U^+ h on backward hops), row by row into this thread's slots uhs[r * bd]
#pragma unroll 1
      for (int ra = 0; ra < 3; ++ra) {
        ff u[6], o[4];
#pragma unroll
        for (int i = 0; i < 6; ++i) u[i] = lsm[hop * 18 + ra * 6 + i];
        su3_row_ff(u, h, o);
        uhs[(0 * 3 + ra) * 2 * bd] = o[0];
        uhs[((0 * 3 + ra) * 2 + 1) * bd] = o[1];
        uhs[(1 * 3 + ra) * 2 * bd] = o[2];
        uhs[((1 * 3 + ra) * 2 + 1) * bd] = o[3];
      }
      // upper spins: acc += uh; lower spins: acc_{2+j} += w'_j uh_{q_j}
#pragma unroll
      for (int r = 0; r < 12; ++r) acc_add(acc[r], uhs[r * bd]);
      const WMul v0 = wmul(w_code(RECON_W, mu, 0, S)), v1 = wmul(w_code(RECON_W, mu, 1, S));
      const int q0 = mu < 2 ? 1 : 0, q1 = 1 - q0;
      const ff* s0 = uhs + (q0 * 6 + (v0.swap ? 1 : 0)) * bd;
      const ff* s1 = uhs + (q1 * 6 + (v1.swap ? 1 : 0)) * bd;
      const int d0 = v0.swap ? -bd : bd, d1 = v1.swap ? -bd : bd;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc_add(acc[(2 * 3 + c) * 2], flip(s0[2 * c * bd], v0.nr));
        acc_add(acc[(2 * 3 + c) * 2 + 1], flip(s0[2 * c * bd + d0], v0.ni));
        acc_add(acc[(3 * 3 + c) * 2], flip(s1[2 * c * bd], v1.nr));
        acc_add(acc[(3 * 3 + c) * 2 + 1], flip(s1[2 * c * bd + d1], v1.ni));
      }
    }
#pragma unroll
    for (int r = 0; r < 24; ++r) acc[r] = fast_two_sum(acc[r].hi, acc[r].lo);
    if (a.alpha != 1.0) {
      const ff al = ff_const(a.alpha);
#pragma unroll
      for (int r = 0; r < 24; ++r) acc[r] = ff_mul(al, acc[r]);
    }
  }

  // ------------------------------------------------------------ epilogue
  char* outb = static_cast<char*>(a.out) + site_offset(site, Lsh, site_bytes);
  const bool pad = s >= Ls;
  if (active && a.pre != PRE_NONE && !pad) {
    const char* auxb = static_cast<const char*>(a.aux) + site_offset(site, Lsh, site_bytes);
    ff o[24];
    if (a.pre == PRE_AUX) {
      load_slice_ff<LSHC>(auxb, s, Lsh, o);
    } else {
      // (Mooee aux)_s = d5 aux_s + c_up aux_{s_up}[upper] + c_lo aux_{s_lo}[lower], c = -1 or m
      const bool dag5 = a.pre == PRE_MOOEE_DAG;
      const int sm = s > 0 ? s - 1 : Ls - 1, sp = s < Ls - 1 ? s + 1 : 0;
      const bool wm = s == 0, wp = s == Ls - 1;  // wrap-around terms carry +m instead of -1
      const int s_up = dag5 ? sp : sm, s_lo = dag5 ? sm : sp;
      const bool w_up = dag5 ? wp : wm, w_lo = dag5 ? wm : wp;
      const ff d5 = ff_const(a.d5), m = ff_const(a.mass);
      load_slice_ff<LSHC>(auxb, s, Lsh, o);
#pragma unroll
      for (int r = 0; r < 24; ++r) o[r] = ff_mul(d5, o[r]);
      ff x[12];
      load_half_ff<LSHC>(auxb, s_up, Lsh, 0, x);
#pragma unroll
      for (int r = 0; r < 12; ++r) o[r] = w_up ? ff_add<+1>(o[r], ff_mul(m, x[r])) : ff_add<-1>(o[r], x[r]);
      load_half_ff<LSHC>(auxb, s_lo, Lsh, 12, x);
#pragma unroll
      for (int r = 0; r < 12; ++r)
        o[12 + r] = w_lo ? ff_add<+1>(o[12 + r], ff_mul(m, x[r])) : ff_add<-1>(o[12 + r], x[r]);
    }
    if (a.beta != 1.0) {
      const ff be = ff_const(a.beta);
#pragma unroll
      for (int r = 0; r < 24; ++r) o[r] = ff_mul(be, o[r]);
    }
#pragma unroll
    for (int r = 0; r < 24; ++r) acc[r] = ff_add<+1>(acc[r], o[r]);
  }
  if (a.post == POST_NONE) {
    if (active) {
      if (pad)
        store_zero_slice<LSHC>(outb, s, Lsh);
      else
        store_slice_ff<LSHC>(outb, s, Lsh, acc);
    }
    return;
  }
  ff* sm = reinterpret_cast<ff*>(smem_raw + (size_t)a.sites_per_cta * (FF_LINK_SITE_BYTES + 32) + FF_UH_BYTES);
  if (active && !pad) {
    ff* dst = sm + ((size_t)site_local * Ls + s) * INV_SLICE_STRIDE;
#pragma unroll
    for (int r = 0; r < 24; ++r) dst[r] = acc[r];
  }
  __syncthreads();
  {
    const int first_site = blockIdx.x * a.sites_per_cta;
    const int nsites = min(a.sites_per_cta, a.g.N4h - first_site);
    const ff m = ff_const(a.mass), inv_d = ff_const(a.inv_d5), inv_den = ff_const(a.inv_den);
    for (int task = tid; task < nsites * 24; task += blockDim.x) {
      const int sl = task / 24;
      const int r = task - sl * 24;
      const bool upper = r < 12;
      const bool forward_form = (a.post == POST_INV) ? upper : !upper;
      mooee_inv_line_ff(sm + (size_t)sl * Ls * INV_SLICE_STRIDE + r, Ls, forward_form, m, inv_d, inv_den);
    }
  }
  __syncthreads();
  if (active) {
    if (pad) {
      store_zero_slice<LSHC>(outb, s, Lsh);
    } else {
      const ff* src = sm + ((size_t)site_local * Ls + s) * INV_SLICE_STRIDE;
#pragma unroll
      for (int r = 0; r < 24; ++r) acc[r] = src[r];
      store_slice_ff<LSHC>(outb, s, Lsh, acc);
    }
  }
}

template <bool DAG, bool C12, int LSC>
cudaError_t launch_ff_one(const DhopArgs& a, int threads, int blocks, size_t smem, cudaStream_t stream) {
  auto kern = dhop_kernel_ff<DAG, C12, LSC>;
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

template <int LSC>
cudaError_t launch_ff_ls(const DhopArgs& a, bool dag, bool c12, int threads, int blocks, size_t smem,
                         cudaStream_t stream) {
  if (dag)
    return c12 ? launch_ff_one<true, true, LSC>(a, threads, blocks, smem, stream)
               : launch_ff_one<true, false, LSC>(a, threads, blocks, smem, stream);
  return c12 ? launch_ff_one<false, true, LSC>(a, threads, blocks, smem, stream)
             : launch_ff_one<false, false, LSC>(a, threads, blocks, smem, stream);
}

}  // namespace

size_t dhop_ff_smem_bytes(int sites_per_cta, int Ls, bool post) {
  return (size_t)sites_per_cta * (FF_LINK_SITE_BYTES + 32) + FF_UH_BYTES +
         (post ? (size_t)sites_per_cta * Ls * INV_SLICE_STRIDE * 8 : 0);
}

cudaError_t launch_dhop_ff(const DhopArgs& a, bool dag, bool c12, int threads, int blocks, size_t smem,
                           cudaStream_t stream) {
  switch (a.g.Ls) {
#define DWF_CASE(L_) \
  case L_:           \
    return launch_ff_ls<L_>(a, dag, c12, threads, blocks, smem, stream);
    DWF_LS_SPECIALISATIONS(DWF_CASE)
#undef DWF_CASE
    default:
      return launch_ff_ls<0>(a, dag, c12, threads, blocks, smem, stream);
  }
}

}  // namespace gdwf
