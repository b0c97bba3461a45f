// Derivative of the action S = |M psi|^2 with respect to the gauge links (the fermion force).
// More generally the kernel differentiates the bilinear -Re chi^+ Dhop psi for any pair of full
// fields (psi, chi), times a coefficient coef (1 for |M psi|^2 with chi = M psi, whose
// variation is 2 Re chi^+ dM psi = -Re chi^+ dDhop psi; -1/2 for the pseudofermion action).
//
// With chi = M psi and M = Mooee - Dhop/2, only the hopping term depends on the links, so per
// link U_mu(x), with phase the boundary factor of the hop x -> x + mu,
//   B1 = sum_{s,spin} psi(x+mu) (x) [(1 - gamma_mu) chi(x)]^+,
//   B2 = sum_{s,spin} psi(x)    (x) [(1 + gamma_mu) chi(x+mu)]^+           (colour outer products),
//   G  = dS/dRe U + i dS/dIm U = -phase (B1^+ + B2)                           (ambient gradient),
//   F  = -TA( phase (-U B1 + B2 U^+) ),  TA(X) = (X - X^+)/2 - tr(X - X^+)/6  (su(3) force),
// so that under U -> exp(eps A) U, A in su(3), dS/deps = Re tr(A^+ F).
// Because (1 -+ gamma_mu)/2 is a rank-2 projector, each spin sum is the sum over the two spins
// of the projected half spinors: sum_spin a (x) [(1 - gamma) b]^+ = sum_{h=0,1} (P a)_h (x) (P b)_h^*.
//
// Thread mapping, as in the hopping kernel: one thread per (4D site, slice pair) for FP32 fields
// and per (4D site, slice) for FP64, whole sites per CTA, one parity per grid row. For each mu the
// threads form their slices' contributions to B1 and B2 of the link U_mu(x) leaving their site
// (the own spinors and the two x + mu neighbours, the same loads as one Dhop hop), the CTA sums
// them over the site's slices through shared memory, and the link algebra is spread over the
// CTA's threads (one 3x3 entry each). FP32 fields: the products are summed in FP32 over blocks of
// at most 8 slice pairs and the block sums in FP64, and the link algebra (U B1, B2 U^+, the
// traceless anti-Hermitian projection) runs in FP32 on those sums: GB300's FP64 pipe is 1/64 of
// its FP32 pipe, and FP64 algebra made the kernel 5x slower for an answer whose error is set by
// the FP32 fields and block sums anyway. FP64 fields use FP64 throughout. F and G are written
// in the canonical FP64 layout [t][z][y][x][mu][3][3].
#include <type_traits>

#include "dhop_kernel.cuh"
#include "ff_arith.cuh"

namespace gdwf {

// Threads per site: slice pairs (FP32, at most 128 for Ls <= 256) or padded slices (FP64; above 128
// slices each thread takes several); sites per CTA fill 128 threads.
inline int force_threads_per_site(int prec, int Ls) {
  const int n = prec == P64 ? ls_padded(Ls) : ls_half(Ls);
  return n < 128 ? n : 128;
}

// Shared memory per site: partial sums of each slice thread (a stride of 37 values, odd, keeps
// the threads' writes in distinct banks), the site's summed B1 and B2 (36), its link (18), Y (18)
// and the output index and boundary phase.
constexpr int FORCE_PART_STRIDE = 37;
inline size_t force_smem_per_site(int prec, int nsg) {
  const size_t v = prec == P64 ? sizeof(double) : sizeof(float);
  return (size_t)nsg * FORCE_PART_STRIDE * v + (36 + 18 + 18) * v + 2 * sizeof(long);
}

// The per-site steps after the slice sums B1, B2 (bsum) of direction mu are in shared memory:
// each site's link, then one (site, a, b) entry per task:
//   G[a][b] = -phase (conj(B1[b][a]) + B2[a][b]),  Y = phase (-U B1 + B2 U^+),
// then F = -TA(Y), TA(Y)[a][b] = (Y[a][b] - conj(Y[b][a]))/2 - delta_ab tr(Y - Y^+)/6.
// A: the arithmetic of the link algebra (double for FP64 fields, float for FP32 fields).
template <int P, bool C12, typename A>
__device__ __forceinline__ void force_site_algebra(int mu, int p, int first, int nsites, const char* Ue, const char* Uo,
                                                   const A* bsum, A* usm, A* ysm, const long* lex_sm,
                                                   const int* ph_sm, double coef, double* F, double* G) {
  using R = typename Store<P>::R;
  constexpr int LB = link_bytes(sizeof(typename Store<P>::T), C12);
  const int tid = threadIdx.x;
  for (int sl = tid; sl < nsites; sl += blockDim.x) {  // the link U_mu(x), third row rebuilt if stored as 12 reals
    R ur[18];
    load_link<P, C12>((p ? Uo : Ue) + ((size_t)(first + sl) * 4 + mu) * LB, ur);
#pragma unroll
    for (int k = 0; k < 18; ++k) usm[(size_t)sl * 18 + k] = (A)ur[k];
  }
  __syncthreads();
  // ---- link algebra, one (site, a, b) entry per task:
  //   G[a][b] = -phase (conj(B1[b][a]) + B2[a][b]),  Y = phase (-U B1 + B2 U^+)
  for (int task = tid; task < nsites * 9; task += blockDim.x) {
    const int sl = task / 9, ab = task - sl * 9, a = ab / 3, b = ab - a * 3;
    const A phd = (A)(coef * (double)ph_sm[sl]);  // F and G are linear in the boundary phase and coef
    const A* B1 = bsum + (size_t)sl * 36;
    const A* B2 = B1 + 18;
    const A* ur = usm + (size_t)sl * 18;
    A yr = 0, yi = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const A ar = ur[(a * 3 + k) * 2], ai = ur[(a * 3 + k) * 2 + 1];
      const A br = B1[(k * 3 + b) * 2], bi = B1[(k * 3 + b) * 2 + 1];
      yr -= ar * br - ai * bi;
      yi -= ar * bi + ai * br;
      const A cr = B2[(a * 3 + k) * 2], ci = B2[(a * 3 + k) * 2 + 1];
      const A dr = ur[(b * 3 + k) * 2], di = -ur[(b * 3 + k) * 2 + 1];  // (U^+)[k][b] = conj(U[b][k])
      yr += cr * dr - ci * di;
      yi += cr * di + ci * dr;
    }
    ysm[(size_t)sl * 18 + ab * 2] = phd * yr;
    ysm[(size_t)sl * 18 + ab * 2 + 1] = phd * yi;
    if (G) {
      double* Go = G + (lex_sm[sl] * 4 + mu) * 18;
      Go[ab * 2] = (double)(-phd * (B1[(b * 3 + a) * 2] + B2[ab * 2]));
      Go[ab * 2 + 1] = (double)(-phd * (-B1[(b * 3 + a) * 2 + 1] + B2[ab * 2 + 1]));
    }
  }
  __syncthreads();
  // ---- F = -TA(Y): TA(Y)[a][b] = (Y[a][b] - conj(Y[b][a]))/2 - delta_ab tr(Y - Y^+)/6
  if (F) {
    for (int task = tid; task < nsites * 9; task += blockDim.x) {
      const int sl = task / 9, ab = task - sl * 9, a = ab / 3, b = ab - a * 3;
      const A* Y = ysm + (size_t)sl * 18;
      const A trim = Y[1] + Y[9] + Y[17];  // Im tr Y; tr(Y - Y^+) = 2 i Im tr Y
      const A tr_ = (A)0.5 * (Y[(a * 3 + b) * 2] - Y[(b * 3 + a) * 2]);
      A ti_ = (A)0.5 * (Y[(a * 3 + b) * 2 + 1] + Y[(b * 3 + a) * 2 + 1]);
      if (a == b) ti_ -= trim / (A)3;
      double* Fo = F + (lex_sm[sl] * 4 + mu) * 18;
      Fo[ab * 2] = -(double)tr_;
      Fo[ab * 2 + 1] = -(double)ti_;
    }
  }
}

template <int P, bool C12>
__global__ void __launch_bounds__(128) k_force(const Geom g, const char* psi, const char* chi, const char* Ue,
                                               const char* Uo, double* F, double* G, double coef, int nsg, int spc) {
  using T = typename Store<P>::T;
  using R = typename Store<P>::R;
  using A = typename std::conditional<P == P64, double, float>::type;  // partial sums and link algebra
  constexpr int LB = link_bytes(sizeof(T), C12);
  constexpr int FLUSH = 8;  // FP32: slice pairs summed in FP32 before an FP64 sum across blocks
  const int Lsh = ls_half(g.Ls);
  const size_t site_bytes = (size_t)Lsh * 2 * 24 * sizeof(T);
  const size_t half_bytes = (size_t)g.N4h * site_bytes;
  // both parities of a block of sites run next to each other, so their shared neighbours are
  // still in L2 when the other parity reads them
  const int p = blockIdx.x & 1;
  const int first = (blockIdx.x >> 1) * spc;
  const int tid = threadIdx.x;
  const int site_local = tid / nsg;
  const int t = tid - site_local * nsg;  // slice pair (FP32) or slice (FP64)
  const int nsites = min(spc, g.N4h - first);
  const bool active = site_local < nsites;
  const int i = first + (active ? site_local : 0);
  int c[4];
  cb_coords(g, i, p, c);
  const char* psi_x = psi + p * half_bytes + site_offset(i, Lsh, site_bytes);
  const char* chi_x = chi + p * half_bytes + site_offset(i, Lsh, site_bytes);

  extern __shared__ __align__(16) unsigned char smem_raw[];
  long* lex_sm = reinterpret_cast<long*>(smem_raw);                          // [spc]
  int* ph_sm = reinterpret_cast<int*>(lex_sm + spc);                         // [spc] (pairs of ints: 8 bytes)
  A* part = reinterpret_cast<A*>(smem_raw + (size_t)spc * 2 * sizeof(long));  // [spc][nsg][37]
  A* bsum = part + (size_t)spc * nsg * FORCE_PART_STRIDE;                      // [spc][36]
  A* usm = bsum + (size_t)spc * 36;                                            // [spc][18]
  A* ysm = usm + (size_t)spc * 18;                                             // [spc][18]
  if (active && t == 0) lex_sm[site_local] = c[0] + (long)g.L[0] * (c[1] + (long)g.L[1] * (c[2] + (long)g.L[2] * c[3]));

#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {  // unrolled: direction-dependent indices stay compile-time
    // ---- this thread's slices: B1 += psi(x+mu) (x) [(1 - gamma) chi(x)]^+, B2 += psi(x) (x) [(1 + gamma) chi(x+mu)]^+
    if (active) {
      int ph;
      const int j = cb_neighbour(g, i, c, mu, true, ph);
      if (t == 0) ph_sm[site_local] = ph;
      const char* psi_f = psi + (1 - p) * half_bytes + site_offset(j, Lsh, site_bytes);
      const char* chi_f = chi + (1 - p) * half_bytes + site_offset(j, Lsh, site_bytes);
      A* dst = part + ((size_t)site_local * nsg + t) * FORCE_PART_STRIDE;
      if constexpr (P == P64) {
        double B[36];
#pragma unroll
        for (int k = 0; k < 36; ++k) B[k] = 0;
        for (int sl5 = t; sl5 < 2 * Lsh; sl5 += nsg) {  // this thread's slices (one unless Ls > 128)
#pragma unroll
          for (int term = 0; term < 2; ++term) {
            double v[24], ha[12], hb[12];
            load_lane64<0>(term == 0 ? psi_f : psi_x, sl5, Lsh, v);
            if (term == 0) project<-1>(mu, v, ha); else project<+1>(mu, v, ha);
            load_lane64<0>(term == 0 ? chi_x : chi_f, sl5, Lsh, v);
            if (term == 0) project<-1>(mu, v, hb); else project<+1>(mu, v, hb);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
              for (int b = 0; b < 3; ++b) {  // sum_h ha[h][a] conj(hb[h][b])
                double re = B[term * 18 + (a * 3 + b) * 2], im = B[term * 18 + (a * 3 + b) * 2 + 1];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const double xr = ha[(h * 3 + a) * 2], xi = ha[(h * 3 + a) * 2 + 1];
                  const double yr = hb[(h * 3 + b) * 2], yi = hb[(h * 3 + b) * 2 + 1];
                  re = fma(xr, yr, fma(xi, yi, re));
                  im = fma(xi, yr, fma(-xr, yi, im));
                }
                B[term * 18 + (a * 3 + b) * 2] = re;
                B[term * 18 + (a * 3 + b) * 2 + 1] = im;
              }
          }
        }
#pragma unroll
        for (int k = 0; k < 36; ++k) dst[k] = B[k];
      } else {
#pragma unroll
        for (int term = 0; term < 2; ++term) {
          float2 v[24], ha[12], hb[12];
          load_pair<P, 0>(term == 0 ? psi_f : psi_x, t, Lsh, v);
          if (term == 0) project2<-1>(mu, v, ha); else project2<+1>(mu, v, ha);
          load_pair<P, 0>(term == 0 ? chi_x : chi_f, t, Lsh, v);
          if (term == 0) project2<-1>(mu, v, hb); else project2<+1>(mu, v, hb);
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {  // both slices of the pair, then their sum
              float2 re = make_float2(0.f, 0.f), im = make_float2(0.f, 0.f);
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const float2 xr = ha[(h * 3 + a) * 2], xi = ha[(h * 3 + a) * 2 + 1];
                const float2 yr = hb[(h * 3 + b) * 2], yi = hb[(h * 3 + b) * 2 + 1];
                re = ffma2(xr, yr, ffma2(xi, yi, re));
                im = ffma2(xi, yr, ffma2(make_float2(-xr.x, -xr.y), yi, im));
              }
              dst[term * 18 + (a * 3 + b) * 2] = re.x + re.y;
              dst[term * 18 + (a * 3 + b) * 2 + 1] = im.x + im.y;
            }
        }
      }
    }
    __syncthreads();
    // ---- sum over the site's slices, one (site, entry) per task; and each site's link
    for (int task = tid; task < nsites * 36; task += blockDim.x) {
      const int sl = task / 36, e = task - sl * 36;
      const A* src = part + (size_t)sl * nsg * FORCE_PART_STRIDE + e;
      A total;
      if constexpr (P == P64) {
        total = 0;
        for (int k = 0; k < nsg; ++k) total += src[(size_t)k * FORCE_PART_STRIDE];
      } else if (nsg <= FLUSH) {  // one block: FP32 throughout
        total = 0.f;
        for (int k = 0; k < nsg; ++k) total += src[(size_t)k * FORCE_PART_STRIDE];
      } else {  // blocks of FLUSH pairs summed in FP64
        double acc = 0;
        for (int k0 = 0; k0 < nsg; k0 += FLUSH) {
          float blk = 0.f;
          const int k1 = min(k0 + FLUSH, nsg);
          for (int k = k0; k < k1; ++k) blk += src[(size_t)k * FORCE_PART_STRIDE];
          acc += (double)blk;
        }
        total = (A)acc;
      }
      bsum[(size_t)sl * 36 + e] = total;
    }
    force_site_algebra<P, C12, A>(mu, p, first, nsites, Ue, Uo, bsum, usm, ysm, lex_sm, ph_sm, coef, F, G);
    __syncthreads();  // shared memory is reused by the next direction
  }
}

// FP32 fields with 8 or 16 slice pairs per site (Ls 15-16, 31-32; the static shared memory of
// fewer pairs per site, i.e. more sites per CTA, would pass 48 KB): a site's
// threads are LSH consecutive lanes of one warp, so the sums over its slices run in registers and
// every synchronisation is within a warp.
//   - Each field is read once as the own site's spinor: the B1 products of all four directions
//     first (own chi(x) held in registers, psi(x + mu) loaded per direction), then the B2 products
//     (own psi(x) held, chi(x + mu) loaded): 10 spinor loads per (site, pair) instead of 16.
//   - The 9 complex products of one (direction, term) are summed over the site's lanes by a
//     butterfly reduce-scatter (xor shuffles; at each level a lane keeps one half of its values
//     and adds its partner's copy of that half), after which lane q holds entries
//     q * NPAD / LSH .. of the site's sum; those go to shared memory.
//   - The link algebra of the site's four links (36 entries) is spread over the same lanes.
// Rounding: the products of a slice pair and the sums over at most 16 pairs are FP32, as in the
// general kernel (which flushes to FP64 after 8 pairs; here 16 pairs at most are summed in FP32).
template <int LSH, int THREADS = 128>
struct ForceRegGeom {
  static constexpr int SPC = THREADS / LSH;                         // sites per CTA
  static constexpr int PER_LANE = (18 + LSH - 1) / LSH;              // sum entries per lane after reduce-scatter
  static constexpr int NPAD = PER_LANE * LSH;                         // 18 reals padded to a multiple of LSH
  // B1 B2 per mu, U per mu, Y per mu, padded so that the sites of a warp fall on different banks:
  // 299 floats give the fewest conflicts of the strides 289-329 over the partial-sum stores and the
  // link algebra's reads of 8-lane sites (53 extra wavefronts per warp against 116 at 289, by
  // simulation; 16-lane sites are indifferent)
  static constexpr int SITE_FLOATS = 4 * 36 + 4 * 18 + 4 * 18 + 11;
};

template <int N, int LSH>
__device__ __forceinline__ void reduce_scatter(float (&v)[N], int lane_in_site) {
  // levels with partner offsets LSH/2, ..., 1: keep the half selected by the offset's bit
#pragma unroll
  for (int off = LSH / 2, len = N / 2; off >= 1; off >>= 1, len >>= 1) {
    const bool upper = (lane_in_site & off) != 0;
#pragma unroll
    for (int k = 0; k < len; ++k) {
      const float send = upper ? v[k] : v[len + k];
      const float keep = upper ? v[len + k] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
}

// The own spinor of a term goes through shared memory and is read back per direction (128
// registers, 4 CTAs per SM): holding it in 48 registers instead needed 168 registers, 3 CTAs per
// SM and some spills, and measured 136 us against 111 us at 16^4 x 16.
template <bool C12, int LSH, int THREADS = 128>
__global__ void __launch_bounds__(THREADS, 512 / THREADS) k_force_reg(const Geom g, const char* psi, const char* chi,
                                                                      const char* Ue, const char* Uo, double* F,
                                                                      double* G, double coef) {
  using GG = ForceRegGeom<LSH, THREADS>;
  constexpr int LB = link_bytes(4, C12);
  constexpr int SPC = GG::SPC, NPAD = GG::NPAD, PER_LANE = GG::PER_LANE;
  const size_t site_bytes = (size_t)LSH * 2 * 24 * 4;
  const size_t half_bytes = (size_t)g.N4h * site_bytes;
  const int p = blockIdx.x & 1;
  const int first = (blockIdx.x >> 1) * SPC;
  const int tid = threadIdx.x;
  const int site_local = tid / LSH;
  const int q = tid - site_local * LSH;  // slice pair, and the lane's place in its site's group
  const bool active = first + site_local < g.N4h;
  const int i = active ? first + site_local : first;  // inactive lanes compute a valid site, store nothing
  int c[4];
  cb_coords(g, i, p, c);
  int nbr[4], phs[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) nbr[mu] = cb_neighbour(g, i, c, mu, true, phs[mu]);

  __shared__ float ssm[SPC][GG::SITE_FLOATS];
  // the own site's spinor of the current term, one 16-byte vector per (chunk, thread): read back
  // for each direction's projection instead of being held in 48 registers
  __shared__ float4 own_sm[12][THREADS];
  float* bs = ssm[site_local];          // [mu][term][18]
  float* us = bs + 4 * 36;              // [mu][18]
  float* ys = us + 4 * 18;              // [mu][18]

  // the site's four links U_mu(x), one per lane (and the third row rebuilt for 12-real links)
  for (int mu = q; mu < 4; mu += LSH) {
    float ur[18];
    load_link<P32, C12>((p ? Uo : Ue) + ((size_t)i * 4 + mu) * LB, ur);
#pragma unroll
    for (int k = 0; k < 18; ++k) us[mu * 18 + k] = ur[k];
  }

#pragma unroll
  for (int term = 0; term < 2; ++term) {
    // term 0: B1 = sum psi(x+mu) (x) [(1 - gamma) chi(x)]^+  (own chi, projector sign -1)
    // term 1: B2 = sum psi(x) (x) [(1 + gamma) chi(x+mu)]^+  (own psi, projector sign +1)
    {
      const char* ob = (term == 0 ? chi : psi) + p * half_bytes + site_offset(i, LSH, site_bytes) + (size_t)q * 16;
#pragma unroll
      for (int k = 0; k < 12; ++k) own_sm[k][tid] = __ldg(reinterpret_cast<const float4*>(ob + k * chunk_stride(LSH)));
    }
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      float2 v[24], ha[12], hb[12];
      load_pair<P32, LSH>((term == 0 ? psi : chi) + (1 - p) * half_bytes + site_offset(nbr[mu], LSH, site_bytes), q,
                          LSH, v);
      {
        float2 own[24];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const float4 t = own_sm[k][tid];
          own[2 * k] = make_float2(t.x, t.y);
          own[2 * k + 1] = make_float2(t.z, t.w);
        }
        if (term == 0)
          project2<-1>(mu, own, hb);
        else
          project2<+1>(mu, own, ha);
      }
      if (term == 0)
        project2<-1>(mu, v, ha);
      else
        project2<+1>(mu, v, hb);
      float s[NPAD];
#pragma unroll
      for (int k = 18; k < NPAD; ++k) s[k] = 0.f;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {  // sum_h ha[h][a] conj(hb[h][b]), both slices of the pair
          float2 re = make_float2(0.f, 0.f), im = make_float2(0.f, 0.f);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float2 xr = ha[(h * 3 + a) * 2], xi = ha[(h * 3 + a) * 2 + 1];
            const float2 yr = hb[(h * 3 + b) * 2], yi = hb[(h * 3 + b) * 2 + 1];
            re = ffma2(xr, yr, ffma2(xi, yi, re));
            im = ffma2(xi, yr, ffma2(make_float2(-xr.x, -xr.y), yi, im));
          }
          s[(a * 3 + b) * 2] = re.x + re.y;
          s[(a * 3 + b) * 2 + 1] = im.x + im.y;
        }
      reduce_scatter<NPAD, LSH>(s, q);
#pragma unroll
      for (int k = 0; k < PER_LANE; ++k) {
        const int e = q * PER_LANE + k;
        if (e < 18) bs[mu * 36 + term * 18 + e] = s[k];
      }
    }
  }
  __syncwarp();
  // link algebra, one (mu, a, b) entry per task over the site's lanes:
  //   G[a][b] = -phase (conj(B1[b][a]) + B2[a][b]),  Y = phase (-U B1 + B2 U^+)
  const long lex = c[0] + (long)g.L[0] * (c[1] + (long)g.L[1] * (c[2] + (long)g.L[2] * c[3]));
  for (int task = q; task < 36; task += LSH) {
    const int mu = task / 9, ab = task - mu * 9, a = ab / 3, b = ab - a * 3;
    const int ph = mu == 0 ? phs[0] : mu == 1 ? phs[1] : mu == 2 ? phs[2] : phs[3];
    const float phd = (float)(coef * (double)ph);
    const float* B1 = bs + mu * 36;
    const float* B2 = B1 + 18;
    const float* ur = us + mu * 18;
    float yr = 0.f, yi = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float ar = ur[(a * 3 + k) * 2], ai = ur[(a * 3 + k) * 2 + 1];
      const float br = B1[(k * 3 + b) * 2], bi = B1[(k * 3 + b) * 2 + 1];
      yr -= ar * br - ai * bi;
      yi -= ar * bi + ai * br;
      const float cr = B2[(a * 3 + k) * 2], ci = B2[(a * 3 + k) * 2 + 1];
      const float dr = ur[(b * 3 + k) * 2], di = -ur[(b * 3 + k) * 2 + 1];  // (U^+)[k][b] = conj(U[b][k])
      yr += cr * dr - ci * di;
      yi += cr * di + ci * dr;
    }
    ys[mu * 18 + ab * 2] = phd * yr;
    ys[mu * 18 + ab * 2 + 1] = phd * yi;
    if (G && active) {
      const double gr = (double)(-phd * (B1[(b * 3 + a) * 2] + B2[ab * 2]));
      const double gi = (double)(-phd * (-B1[(b * 3 + a) * 2 + 1] + B2[ab * 2 + 1]));
      *reinterpret_cast<double2*>(G + (lex * 4 + mu) * 18 + ab * 2) = make_double2(gr, gi);
    }
  }
  __syncwarp();
  // F = -TA(Y): TA(Y)[a][b] = (Y[a][b] - conj(Y[b][a]))/2 - delta_ab tr(Y - Y^+)/6
  if (F && active) {
    for (int task = q; task < 36; task += LSH) {
      const int mu = task / 9, ab = task - mu * 9, a = ab / 3, b = ab - a * 3;
      const float* Y = ys + mu * 18;
      const float trim = Y[1] + Y[9] + Y[17];  // Im tr Y; tr(Y - Y^+) = 2 i Im tr Y
      const float tr_ = 0.5f * (Y[(a * 3 + b) * 2] - Y[(b * 3 + a) * 2]);
      float ti_ = 0.5f * (Y[(a * 3 + b) * 2 + 1] + Y[(b * 3 + a) * 2 + 1]);
      if (a == b) ti_ -= trim / 3.f;
      *reinterpret_cast<double2*>(F + (lex * 4 + mu) * 18 + ab * 2) = make_double2(-(double)tr_, -(double)ti_);
    }
  }
}

// FP64 fields in float-float arithmetic (the handle's FP64 arithmetic set to float-float): the
// per-slice products in pairs of FP32 numbers, the slice sums in float-float, then the site's
// sums rounded to FP64 for the (per 4D site, cheap) link algebra. One thread per (site, slice)
// (Ls <= 128, so one slice each); the direction loop is not unrolled, and the projections read
// their direction-dependent parts by address, so that one short code path serves every mu (the
// unrolled float-float code would overflow the instruction cache, as in the hopping kernel).
template <bool C12>
__global__ void __launch_bounds__(128) k_force_ff(const Geom g, const char* psi, const char* chi, const char* Ue,
                                                  const char* Uo, double* F, double* G, double coef, int nsg,
                                                  int spc) {
  using namespace ffa;
  const int Lsh = ls_half(g.Ls);
  const size_t site_bytes = (size_t)Lsh * 2 * 24 * 8;
  const size_t half_bytes = (size_t)g.N4h * site_bytes;
  const size_t cs = chunk_stride(Lsh);
  const int p = blockIdx.x & 1;
  const int first = (blockIdx.x >> 1) * spc;
  const int tid = threadIdx.x;
  const int site_local = tid / nsg;
  const int t = tid - site_local * nsg;  // the thread's slice
  const int nsites = min(spc, g.N4h - first);
  const bool active = site_local < nsites;
  const int i = first + (active ? site_local : 0);
  int c[4];
  cb_coords(g, i, p, c);
  const char* psi_x = psi + p * half_bytes + site_offset(i, Lsh, site_bytes) + (size_t)t * 8;
  const char* chi_x = chi + p * half_bytes + site_offset(i, Lsh, site_bytes) + (size_t)t * 8;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  long* lex_sm = reinterpret_cast<long*>(smem_raw);
  int* ph_sm = reinterpret_cast<int*>(lex_sm + spc);
  ff* part = reinterpret_cast<ff*>(smem_raw + (size_t)spc * 2 * sizeof(long));  // [spc][nsg][37] (S, E) pairs
  double* bsum = reinterpret_cast<double*>(part + (size_t)spc * nsg * FORCE_PART_STRIDE);  // [spc][36]
  double* usm = bsum + (size_t)spc * 36;
  double* ysm = usm + (size_t)spc * 18;
  if (active && t == 0) lex_sm[site_local] = c[0] + (long)g.L[0] * (c[1] + (long)g.L[1] * (c[2] + (long)g.L[2] * c[3]));
  // forward neighbours and phases at compile-time mu (a runtime mu would index c and g through
  // local memory), picked by selects in the rolled loop below
  int nf[4], pf[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) nf[m] = cb_neighbour(g, i, c, m, true, pf[m]);

#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    if (active) {
      const int j = mu == 0 ? nf[0] : mu == 1 ? nf[1] : mu == 2 ? nf[2] : nf[3];
      const int ph = mu == 0 ? pf[0] : mu == 1 ? pf[1] : mu == 2 ? pf[2] : pf[3];
      if (t == 0) ph_sm[site_local] = ph;
      const size_t jo = (1 - p) * half_bytes + site_offset(j, Lsh, site_bytes) + (size_t)t * 8;
      ff* dst = part + ((size_t)site_local * nsg + t) * FORCE_PART_STRIDE;
      // term 0: B1 = psi(x+mu) (x) [(1 - gamma) chi(x)]^+;  term 1: B2 = psi(x) (x) [(1 + gamma) chi(x+mu)]^+
#pragma unroll 1
      for (int term = 0; term < 2; ++term) {
        const int S = term == 0 ? -1 : +1;
        ff ha[12], hb[12];
        project_load_ff(term == 0 ? psi + jo : psi_x, mu, S, cs, ha);
        project_load_ff(term == 0 ? chi_x : chi + jo, mu, S, cs, hb);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) {  // sum_h ha[h][a] conj(hb[h][b])
            ffacc re, im;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              const ff xr = ha[(hh * 3 + a) * 2], xi = ha[(hh * 3 + a) * 2 + 1];
              const ff yr = hb[(hh * 3 + b) * 2], yi = hb[(hh * 3 + b) * 2 + 1];
              if (hh == 0) {
                dot_first(re, xr, yr, false);
                dot_first(im, xi, yr, false);
              } else {
                dot_add<+1>(re, xr, yr);
                dot_add<+1>(im, xi, yr);
              }
              dot_add<+1>(re, xi, yi);
              dot_add<-1>(im, xr, yi);
            }
            dst[term * 18 + (a * 3 + b) * 2] = ff_make(re.s, re.e);
            dst[term * 18 + (a * 3 + b) * 2 + 1] = ff_make(im.s, im.e);
          }
      }
    }
    __syncthreads();
    // ---- sum over the site's slices in float-float, one (site, entry) per task, rounded to FP64
    for (int task = tid; task < nsites * 36; task += blockDim.x) {
      const int sl = task / 36, e = task - sl * 36;
      const ff* src = part + (size_t)sl * nsg * FORCE_PART_STRIDE + e;
      ff total = ff_make(0.f, 0.f);
      for (int k = 0; k < nsg; ++k) acc_add(total, src[(size_t)k * FORCE_PART_STRIDE]);
      bsum[(size_t)sl * 36 + e] = ff_to_double(fast_two_sum(total.hi, total.lo));
    }
    force_site_algebra<P64, C12, double>(mu, p, first, nsites, Ue, Uo, bsum, usm, ysm, lex_sm, ph_sm, coef, F, G);
    __syncthreads();  // shared memory is reused by the next direction
  }
}

cudaError_t launch_force(int prec, bool c12, const Geom& g, const void* psi, const void* chi, const void* Ue,
                         const void* Uo, double* F, double* G, double coef, bool float_float, cudaStream_t st) {
  const int nsg = force_threads_per_site(prec, g.Ls);
  const size_t per_site = force_smem_per_site(prec, nsg);
  int spc = 128 / nsg;
  if ((size_t)spc * per_site > 48 * 1024) spc = (int)(48 * 1024 / per_site);  // short Ls: many sites per CTA
  if (spc < 1) spc = 1;
  const int threads = nsg * spc;
  const dim3 grid((unsigned)(2 * ((g.N4h + spc - 1) / spc)));  // (site block, parity), parity fastest
  const size_t smem = (size_t)spc * per_site;
  const char* ps = static_cast<const char*>(psi);
  const char* ch = static_cast<const char*>(chi);
  const char* e = static_cast<const char*>(Ue);
  const char* o = static_cast<const char*>(Uo);
#define FK(P_)                                                                                 \
  if (c12)                                                                                     \
    k_force<P_, true><<<grid, threads, smem, st>>>(g, ps, ch, e, o, F, G, coef, nsg, spc);    \
  else                                                                                         \
    k_force<P_, false><<<grid, threads, smem, st>>>(g, ps, ch, e, o, F, G, coef, nsg, spc);
  if (prec == P64 && float_float) {
    if (c12)
      k_force_ff<true><<<grid, threads, smem, st>>>(g, ps, ch, e, o, F, G, coef, nsg, spc);
    else
      k_force_ff<false><<<grid, threads, smem, st>>>(g, ps, ch, e, o, F, G, coef, nsg, spc);
    return cudaGetLastError();
  }
  const int Lsh = ls_half(g.Ls);
  if (prec == P32 && (Lsh == 8 || Lsh == 16)) {
    // CTAs of 64 threads for 8 pairs per site (8 sites; measured 108.2 us against 109.5 us with
    // 128 threads at 16^4 x 16, the same warps per SM and a finer last wave), 128 for 16 pairs
#define FR(L_, T_)                                                                                       \
  {                                                                                                      \
    constexpr int spc = ForceRegGeom<L_, T_>::SPC;                                                       \
    const dim3 gr((unsigned)(2 * ((g.N4h + spc - 1) / spc)));                                            \
    if (c12)                                                                                             \
      k_force_reg<true, L_, T_><<<gr, T_, 0, st>>>(g, ps, ch, e, o, F, G, coef);                         \
    else                                                                                                 \
      k_force_reg<false, L_, T_><<<gr, T_, 0, st>>>(g, ps, ch, e, o, F, G, coef);                        \
  }
    if (Lsh == 8) FR(8, 64) else FR(16, 128)
#undef FR
    return cudaGetLastError();
  }
  switch (prec) {
    case P64: FK(P64) break;
    case P32: FK(P32) break;
    default: return cudaErrorInvalidValue;
  }
#undef FK
  return cudaGetLastError();
}

}  // namespace gdwf
