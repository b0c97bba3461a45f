// The Wilson hopping stencil on 5D domain-wall fields (DhopEO / DhopOE and their adjoints),
// with optional fused fifth-dimension epilogues.
//
// The paper (Section 3, the Nsight-Compute profile of "the main kernel DWF code"; Conclusion,
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
// Thread mapping: one thread per (4D checkerboard site, s-group); a site's Ls slices are split
// into nsg = Ls / ST groups and thread sg handles s = sg, sg + nsg, ..., so that the lanes of a
// warp read consecutive 16-byte vectors of the neighbour's site block. All threads of a site
// load the same link (a broadcast load), so every link is read from memory once per site and
// reused for all Ls slices; a CTA holds whole sites, which the fused Mooee^-1 epilogue needs.
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
  int nsg;            // s-groups per site
  int sites_per_cta;  // whole sites per CTA
  int pre, post;
  double alpha, beta;
  double d5;       // 5 - M5
  double mass;     // m
  double inv_d5;   // 1 / (5 - M5)
  double inv_den;  // 1 / ((5 - M5) + m (5 - M5)^-(Ls-1))
  int seg;         // > 0: bulk-copy staged kernel with this many sites per CTA (dhop_tma.cuh)
  int* status;     // device status word: bit 0 set if a staged kernel's wait timed out
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

template <int P, int LSC = 0>
__device__ __forceinline__ void load_spinor(const char* site_block, int s, int Ls_rt, typename Store<P>::R* psi) {
  constexpr int VEC = Store<P>::VEC;
  constexpr int NCH = 24 / VEC;
  const int Ls = LSC > 0 ? LSC : Ls_rt;
  const char* b = site_block + (size_t)s * 16;
#pragma unroll
  for (int k = 0; k < NCH; ++k) ld16<P>(b + (size_t)k * Ls * 16, psi + k * VEC);
}

template <int P, int LSC = 0>
__device__ __forceinline__ void store_spinor(char* site_block, int s, int Ls_rt, const typename Store<P>::R* v) {
  constexpr int VEC = Store<P>::VEC;
  constexpr int NCH = 24 / VEC;
  const int Ls = LSC > 0 ? LSC : Ls_rt;
  char* b = site_block + (size_t)s * 16;
#pragma unroll
  for (int k = 0; k < NCH; ++k) st16<P>(b + (size_t)k * Ls * 16, v + k * VEC);
}

// The same two loads from shared memory (plain loads; the staged kernel reads its own buffers).
template <int P, int LSC>
__device__ __forceinline__ void load_spinor_smem(const char* site_block, int s, typename Store<P>::R* psi) {
  constexpr int VEC = Store<P>::VEC;
  constexpr int NCH = 24 / VEC;
  const char* b = site_block + (size_t)s * 16;
#pragma unroll
  for (int k = 0; k < NCH; ++k) ld16c<P>(b + (size_t)k * LSC * 16, psi + k * VEC);
}

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

// (Mooee aux)_s or (Mooee^+ aux)_s for one slice: the upper (P+) reals couple to s-1 and the
// lower (P-) reals to s+1, with +m replacing -1 on the wrap-around; the adjoint swaps them.
template <int P, bool DAG5>
__device__ __forceinline__ void mooee_slice(const char* site_block, int s, int Ls, double d5, double mass,
                                            typename Store<P>::R* o) {
  using R = typename Store<P>::R;
  constexpr int VEC = Store<P>::VEC;
  constexpr int NCH = 24 / VEC;
  const int sm = s > 0 ? s - 1 : Ls - 1;
  const int sp = s < Ls - 1 ? s + 1 : 0;
  const R cm = s > 0 ? R(-1) : R(mass);
  const R cp = s < Ls - 1 ? R(-1) : R(mass);
  // upper reals use (s_up, c_up), lower reals use (s_lo, c_lo)
  const int s_up = DAG5 ? sp : sm, s_lo = DAG5 ? sm : sp;
  const R c_up = DAG5 ? cp : cm, c_lo = DAG5 ? cm : cp;
  const R d = R(d5);
#pragma unroll
  for (int k = 0; k < NCH; ++k) {
    R self[VEC], up[VEC], lo[VEC];
    ld16<P>(site_block + ((size_t)k * Ls + s) * 16, self);
    const bool need_up = k * VEC < 12;
    const bool need_lo = (k + 1) * VEC > 12;
    if (need_up) ld16<P>(site_block + ((size_t)k * Ls + s_up) * 16, up);
    if (need_lo) ld16<P>(site_block + ((size_t)k * Ls + s_lo) * 16, lo);
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const int r = k * VEC + v;
      o[r] = d * self[v] + (r < 12 ? c_up * up[v] : c_lo * lo[v]);
    }
  }
}

// In-place inverse of the fifth-dimension matrix along one real component of one site, held
// in shared memory with stride 24 between slices. FORWARD_FORM solves the chirality coupled to
// s-1: y_0 = (b_0 - m sum_{k>=1} d^-(Ls-k) b_k) / (d + m d^-(Ls-1)), y_s = (b_s + y_{s-1}) / d;
// otherwise the mirror image in s.
template <typename R>
__device__ __forceinline__ void mooee_inv_line(R* v, int Ls, bool forward_form, R mass, R inv_d, R inv_den) {
  if (forward_form) {
    R acc = 0;
    for (int k = 1; k < Ls; ++k) acc = (acc + v[k * 24]) * inv_d;
    R y = (v[0] - mass * acc) * inv_den;
    v[0] = y;
    for (int s = 1; s < Ls; ++s) {
      y = (v[s * 24] + y) * inv_d;
      v[s * 24] = y;
    }
  } else {
    R acc = 0;
    for (int k = Ls - 2; k >= 0; --k) acc = (acc + v[k * 24]) * inv_d;
    R y = (v[(Ls - 1) * 24] - mass * acc) * inv_den;
    v[(Ls - 1) * 24] = y;
    for (int s = Ls - 2; s >= 0; --s) {
      y = (v[s * 24] + y) * inv_d;
      v[s * 24] = y;
    }
  }
}

template <int P, int ST, bool DAG, bool C12, int LSC>
__device__ __forceinline__ void dhop_body(const DhopArgs& a) {
  using T = typename Store<P>::T;
  using R = typename Store<P>::R;
  constexpr int LB = link_bytes(sizeof(T), C12);
  constexpr int SF = DAG ? +1 : -1;  // forward projector (1 + SF gamma)
  constexpr int SB = -SF;            // backward projector
  const int Ls = LSC > 0 ? LSC : a.g.Ls;
  const int nsg = LSC > 0 ? LSC / ST : a.nsg;
  const int tid = threadIdx.x;
  const int site_local = tid / nsg;
  const int sg = tid - site_local * nsg;
  const int site = blockIdx.x * a.sites_per_cta + site_local;
  const bool active = site_local < a.sites_per_cta && site < a.g.N4h;
  const size_t site_bytes = (size_t)Ls * 24 * sizeof(T);
  const R alpha = R(a.alpha);

  R acc[ST][24];
#pragma unroll
  for (int k = 0; k < ST; ++k)
#pragma unroll
    for (int r = 0; r < 24; ++r) acc[k][r] = 0;

  if (active) {
    int c[4];
    cb_coords(a.g, site, a.out_parity, c);
    const char* in = static_cast<const char*>(a.in);
    const char* Uo = static_cast<const char*>(a.Uout);
    const char* Ui = static_cast<const char*>(a.Uin);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      {  // forward hop: (1 + SF gamma_mu) U_mu(x) psi(x + mu)
        int ph;
        const int j = cb_neighbour(a.g, site, c, mu, true, ph);
        R u[18];
        load_link<P, C12>(Uo + ((size_t)site * 4 + mu) * LB, u);
        const char* pj = in + (size_t)j * site_bytes;
        const R scale = ph < 0 ? -alpha : alpha;
#pragma unroll
        for (int k = 0; k < ST; ++k) {
          R psi[24], h[12], uh[12];
          load_spinor<P, LSC>(pj, sg + k * nsg, Ls, psi);
          project<SF>(mu, psi, h);
          su3_mul<false>(u, h, uh);
          accumulate<SF>(mu, uh, scale, acc[k]);
        }
      }
      {  // backward hop: (1 + SB gamma_mu) U_mu(x - mu)^+ psi(x - mu)
        int ph;
        const int j = cb_neighbour(a.g, site, c, mu, false, ph);
        R u[18];
        load_link<P, C12>(Ui + ((size_t)j * 4 + mu) * LB, u);
        const char* pj = in + (size_t)j * site_bytes;
        const R scale = ph < 0 ? -alpha : alpha;
#pragma unroll
        for (int k = 0; k < ST; ++k) {
          R psi[24], h[12], uh[12];
          load_spinor<P, LSC>(pj, sg + k * nsg, Ls, psi);
          project<SB>(mu, psi, h);
          su3_mul<true>(u, h, uh);
          accumulate<SB>(mu, uh, scale, acc[k]);
        }
      }
    }
  }

  // ------------------------------------------------------------ epilogue
  const R beta = R(a.beta);
  const char* auxb = a.pre != PRE_NONE ? static_cast<const char*>(a.aux) + (size_t)site * site_bytes : nullptr;
  char* outb = static_cast<char*>(a.out) + (size_t)site * site_bytes;
  if (active && a.pre != PRE_NONE) {
#pragma unroll
    for (int k = 0; k < ST; ++k) {
      const int s = sg + k * nsg;
      R o[24];
      if (a.pre == PRE_AUX)
        load_spinor<P, LSC>(auxb, s, Ls, o);
      else if (a.pre == PRE_MOOEE)
        mooee_slice<P, false>(auxb, s, Ls, a.d5, a.mass, o);
      else
        mooee_slice<P, true>(auxb, s, Ls, a.d5, a.mass, o);
#pragma unroll
      for (int r = 0; r < 24; ++r) acc[k][r] = fma_r(beta, o[r], acc[k][r]);
    }
  }
  if (a.post == POST_NONE) {
    if (active) {
#pragma unroll
      for (int k = 0; k < ST; ++k) store_spinor<P, LSC>(outb, sg + k * nsg, Ls, acc[k]);
    }
    return;
  }
  // Fifth-dimension inverse through shared memory: whole sites live in this CTA.
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  if (active) {
#pragma unroll
    for (int k = 0; k < ST; ++k) {
      R* dst = sm + ((size_t)site_local * Ls + sg + k * nsg) * 24;
#pragma unroll
      for (int r = 0; r < 24; ++r) dst[r] = acc[k][r];
    }
  }
  __syncthreads();
  const int first_site = blockIdx.x * a.sites_per_cta;
  const int nsites = min(a.sites_per_cta, a.g.N4h - first_site);
  for (int task = tid; task < nsites * 24; task += blockDim.x) {
    const int sl = task / 24;
    const int r = task - sl * 24;
    const bool upper = r < 12;
    const bool forward_form = (a.post == POST_INV) ? upper : !upper;
    mooee_inv_line<R>(sm + (size_t)sl * Ls * 24 + r, Ls, forward_form, R(a.mass), R(a.inv_d5), R(a.inv_den));
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int k = 0; k < ST; ++k) {
      const int s = sg + k * nsg;
      store_spinor<P, LSC>(outb, s, Ls, sm + ((size_t)site_local * Ls + s) * 24);
    }
  }
}

// Register budget: at most 256 threads per CTA and two such CTAs per SM (128 registers per
// thread): the measured optimum for the FP32 and 16-bit kernels on GB300 (more resident warps
// with fewer registers spill and run slower). The FP64 kernel is bound by the FP64 pipe and
// keeps more registers instead.
template <int P>
struct DhopOccupancy {
  static constexpr int MIN_BLOCKS = (P == P64) ? 1 : 2;
};

// Slices per thread: two for the 16-bit storage formats at a compile-time Ls (halves the link
// loads and conversions per slice), one otherwise.
__host__ __device__ constexpr int dhop_slices_per_thread(int prec, int lsc) {
  return (lsc > 0 && (prec == P16 || prec == PB16)) ? 2 : 1;
}

// Ls values with a compile-time specialisation; any other Ls runs the generic kernel (LSC = 0).
#define DWF_LS_SPECIALISATIONS(M) M(8) M(12) M(16) M(24) M(32)
inline bool dhop_ls_specialised(int Ls) { return Ls == 8 || Ls == 12 || Ls == 16 || Ls == 24 || Ls == 32; }

template <int P, int ST, bool DAG, bool C12, int LSC>
__global__ void __launch_bounds__(256, DhopOccupancy<P>::MIN_BLOCKS) dhop_kernel(const __grid_constant__ DhopArgs a) {
  dhop_body<P, ST, DAG, C12, LSC>(a);
}

template <int P>
cudaError_t launch_dhop(const DhopArgs& a, int st, bool dag, bool c12, int threads, int blocks, size_t smem,
                        cudaStream_t stream);
template <>
cudaError_t launch_dhop<P64>(const DhopArgs&, int, bool, bool, int, int, size_t, cudaStream_t);
template <>
cudaError_t launch_dhop<P32>(const DhopArgs&, int, bool, bool, int, int, size_t, cudaStream_t);
template <>
cudaError_t launch_dhop<P16>(const DhopArgs&, int, bool, bool, int, int, size_t, cudaStream_t);
template <>
cudaError_t launch_dhop<PB16>(const DhopArgs&, int, bool, bool, int, int, size_t, cudaStream_t);

}  // namespace gdwf
