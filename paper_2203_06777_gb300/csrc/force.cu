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
// Thread mapping: one thread per link (x, mu), looping over the slices. FP32 fields: each slice
// pair is projected and multiplied in packed FP32x2 arithmetic and summed in FP32 over blocks of
// at most 8 pairs, each block then added into FP64 accumulators (GB300's FP64 pipe is 1/64 of
// FP32, so per-pair FP64 adds would dominate the kernel); FP64 fields use FP64 throughout. The link algebra (U B1, B2 U^+, the traceless anti-Hermitian projection) is FP64,
// and F and G are written in the canonical FP64 layout [t][z][y][x][mu][3][3].
#include "dhop_kernel.cuh"

namespace gdwf {

template <int P, bool C12>
__global__ void __launch_bounds__(128) k_force(const Geom g, const char* psi, const char* chi, const char* Ue,
                                               const char* Uo, double* F, double* G, double coef) {
  using T = typename Store<P>::T;
  using R = typename Store<P>::R;
  constexpr int LB = link_bytes(sizeof(T), C12);
  const int Ls = g.Ls;
  const int Lsh = ls_half(Ls);
  const size_t site_bytes = (size_t)Lsh * 2 * 24 * sizeof(T);
  const size_t half_bytes = (size_t)g.N4h * site_bytes;
  const long link = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (link >= 8L * g.N4h) return;
  const int mu = (int)(link & 3);
  const long rest = link >> 2;
  const int p = rest >= g.N4h ? 1 : 0;
  const int i = (int)(rest - (long)p * g.N4h);
  int c[4];
  cb_coords(g, i, p, c);
  int ph;
  const int j = cb_neighbour(g, i, c, mu, true, ph);
  const char* psi_x = psi + p * half_bytes + (size_t)i * site_bytes;
  const char* chi_x = chi + p * half_bytes + (size_t)i * site_bytes;
  const char* psi_f = psi + (1 - p) * half_bytes + (size_t)j * site_bytes;
  const char* chi_f = chi + (1 - p) * half_bytes + (size_t)j * site_bytes;

  double B1[18], B2[18];
#pragma unroll
  for (int k = 0; k < 18; ++k) B1[k] = B2[k] = 0.0;
  if constexpr (P == P64) {
#pragma unroll
    for (int term = 0; term < 2; ++term) {
      double* B = term == 0 ? B1 : B2;
      const char* fa = term == 0 ? psi_f : psi_x;
      const char* fb = term == 0 ? chi_x : chi_f;
      for (int s = 0; s < Ls; ++s) {
        double v[24], ha[12], hb[12];
        load_lane64<0>(fa, s, Lsh, v);
        if (term == 0) project<-1>(mu, v, ha); else project<+1>(mu, v, ha);
        load_lane64<0>(fb, s, Lsh, v);
        if (term == 0) project<-1>(mu, v, hb); else project<+1>(mu, v, hb);
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {  // B[a][b] += ha[h][a] conj(hb[h][b])
              const double xr = ha[(h * 3 + a) * 2], xi = ha[(h * 3 + a) * 2 + 1];
              const double yr = hb[(h * 3 + b) * 2], yi = hb[(h * 3 + b) * 2 + 1];
              B[(a * 3 + b) * 2] = fma(xr, yr, fma(xi, yi, B[(a * 3 + b) * 2]));
              B[(a * 3 + b) * 2 + 1] = fma(xi, yr, fma(-xr, yi, B[(a * 3 + b) * 2 + 1]));
            }
      }
    }
  } else {
    // Pad slices are zero in every field, so pairs are used whole. Each term is summed in
    // FP32x2 (one lane per slice parity) over blocks of up to FLUSH pairs, and each block's two
    // lanes are added into the FP64 accumulators: at most 2 FLUSH FP32 terms per rounding chain.
    constexpr int FLUSH = 8;
#pragma unroll
    for (int term = 0; term < 2; ++term) {
      double* B = term == 0 ? B1 : B2;
      const char* fa = term == 0 ? psi_f : psi_x;
      const char* fb = term == 0 ? chi_x : chi_f;
      for (int q0 = 0; q0 < Lsh; q0 += FLUSH) {
        float2 acc[18];
#pragma unroll
        for (int k = 0; k < 18; ++k) acc[k] = make_float2(0.f, 0.f);
        const int q1 = min(q0 + FLUSH, Lsh);
        for (int q = q0; q < q1; ++q) {
          float2 v[24], ha[12], hb[12];
          load_pair<P, 0>(fa, q, Lsh, v);
          if (term == 0) project2<-1>(mu, v, ha); else project2<+1>(mu, v, ha);
          load_pair<P, 0>(fb, q, Lsh, v);
          if (term == 0) project2<-1>(mu, v, hb); else project2<+1>(mu, v, hb);
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
              for (int b = 0; b < 3; ++b) {  // acc[a][b] += ha[h][a] conj(hb[h][b])
                const float2 xr = ha[(h * 3 + a) * 2], xi = ha[(h * 3 + a) * 2 + 1];
                const float2 yr = hb[(h * 3 + b) * 2], yi = hb[(h * 3 + b) * 2 + 1];
                acc[(a * 3 + b) * 2] = ffma2(xr, yr, ffma2(xi, yi, acc[(a * 3 + b) * 2]));
                acc[(a * 3 + b) * 2 + 1] =
                    ffma2(xi, yr, ffma2(make_float2(-xr.x, -xr.y), yi, acc[(a * 3 + b) * 2 + 1]));
              }
        }
#pragma unroll
        for (int k = 0; k < 18; ++k) B[k] += (double)acc[k].x + (double)acc[k].y;
      }
    }
  }

  R ur[18];
  load_link<P, C12>((p ? Uo : Ue) + ((size_t)i * 4 + mu) * LB, ur);
  double u[18];
#pragma unroll
  for (int k = 0; k < 18; ++k) u[k] = (double)ur[k];
  const double phd = coef * (double)ph;  // F and G are linear in the boundary phase and coef
  const long lex = c[0] + (long)g.L[0] * (c[1] + (long)g.L[1] * (c[2] + (long)g.L[2] * c[3]));
  double* Fo = F ? F + (lex * 4 + mu) * 18 : nullptr;
  double* Go = G ? G + (lex * 4 + mu) * 18 : nullptr;
  if (Go) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {  // G[a][b] = -phase (conj(B1[b][a]) + B2[a][b])
        Go[(a * 3 + b) * 2] = -phd * (B1[(b * 3 + a) * 2] + B2[(a * 3 + b) * 2]);
        Go[(a * 3 + b) * 2 + 1] = -phd * (-B1[(b * 3 + a) * 2 + 1] + B2[(a * 3 + b) * 2 + 1]);
      }
  }
  if (Fo) {
    double Y[18];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {  // Y = phase (-U B1 + B2 U^+)
        double yr = 0, yi = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double ar = u[(a * 3 + k) * 2], ai = u[(a * 3 + k) * 2 + 1];
          const double br = B1[(k * 3 + b) * 2], bi = B1[(k * 3 + b) * 2 + 1];
          yr -= ar * br - ai * bi;
          yi -= ar * bi + ai * br;
          const double cr = B2[(a * 3 + k) * 2], ci = B2[(a * 3 + k) * 2 + 1];
          const double dr = u[(b * 3 + k) * 2], di = -u[(b * 3 + k) * 2 + 1];  // (U^+)[k][b] = conj(U[b][k])
          yr += cr * dr - ci * di;
          yi += cr * di + ci * dr;
        }
        Y[(a * 3 + b) * 2] = phd * yr;
        Y[(a * 3 + b) * 2 + 1] = phd * yi;
      }
    // F = -TA(Y): TA(Y)[a][b] = (Y[a][b] - conj(Y[b][a]))/2 - delta_ab tr(Y - Y^+)/6
    const double trim = (Y[1] + Y[9] + Y[17]);  // Im tr Y; tr(Y - Y^+) = 2 i Im tr Y
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        double tr_ = 0.5 * (Y[(a * 3 + b) * 2] - Y[(b * 3 + a) * 2]);
        double ti_ = 0.5 * (Y[(a * 3 + b) * 2 + 1] + Y[(b * 3 + a) * 2 + 1]);
        if (a == b) ti_ -= trim / 3.0;
        Fo[(a * 3 + b) * 2] = -tr_;
        Fo[(a * 3 + b) * 2 + 1] = -ti_;
      }
  }
}

cudaError_t launch_force(int prec, bool c12, const Geom& g, const void* psi, const void* chi, const void* Ue,
                         const void* Uo, double* F, double* G, double coef, cudaStream_t st) {
  const int threads = 128;
  const long links = 8L * g.N4h;
  const int blocks = (int)((links + threads - 1) / threads);
  const char* ps = static_cast<const char*>(psi);
  const char* ch = static_cast<const char*>(chi);
  const char* e = static_cast<const char*>(Ue);
  const char* o = static_cast<const char*>(Uo);
#define FK(P_)                                                                   \
  if (c12)                                                                       \
    k_force<P_, true><<<blocks, threads, 0, st>>>(g, ps, ch, e, o, F, G, coef);        \
  else                                                                           \
    k_force<P_, false><<<blocks, threads, 0, st>>>(g, ps, ch, e, o, F, G, coef);
  switch (prec) {
    case P64: FK(P64) break;
    case P32: FK(P32) break;
    default: return cudaErrorInvalidValue;
  }
#undef FK
  return cudaGetLastError();
}

}  // namespace gdwf
