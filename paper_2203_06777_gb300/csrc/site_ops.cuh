// Site-local kernels of the library: layout conversion (pack/unpack of spinors and links),
// precision conversion, the standalone fifth-dimension operators Mooee / Mooee^-1, the
// FP64-accumulated reductions and the CG vector updates. Launchers are declared here and
// defined in site_ops.cu.
#pragma once

#include "dwf_common.cuh"

namespace gdwf {

// Scalars of a CG solve, kept in device memory so that iterations need no host round trip.
enum CgScalar : int {
  S_RR = 0,     // |r|^2 of the current residual
  S_PAP = 1,    // <p, A p>
  S_ALPHA = 2,  // rr / pAp
  S_BETA = 3,   // rr_new / rr (times the p rescale factor)
  S_RRNEW = 4,  // |r_new|^2
  S_PSCALE = 5, // factor applied to p in the next p update (rescaling of the sloppy vectors)
  S_TMP0 = 6,
  S_TMP1 = 7,
  S_RROLD = 8,  // |r|^2 before the last FIN_BETA (the denominator of its beta)
  S_COUNT = 16
};

// Fixed reduction geometry: the partial-sum layout, and hence the summation order, never
// depends on the data, so results are bitwise reproducible.
constexpr int RED_BLOCKS = 608;  // 4 x 152 SMs
constexpr int RED_THREADS = 256;

// Finalise kinds: what the single-CTA second pass does with the total.
enum FinalKind : int {
  FIN_STORE = 0,  // scal[dst] = total (and scal[dst+1] = imaginary part for inner products)
  FIN_ALPHA = 1,  // scal[S_PAP] = total; scal[S_ALPHA] = scal[S_RR] / total
  FIN_BETA = 2,   // scal[S_RRNEW] = total; scal[S_BETA] = scal[S_PSCALE] * total / scal[S_RR];
                  // scal[S_RROLD] = scal[S_RR]; scal[S_RR] = total
};

// Second pass over n partial sums (one component) in a fixed order, finalised as `kind`: for the
// per-CTA sums of the hopping kernel's CG epilogues.
cudaError_t launch_finalize_n(const double* partials, int n, double* scal, int kind, int dst, cudaStream_t st);

cudaError_t launch_pack_spinor(int prec, const Geom& g, const double* canon, void* field, int subset, bool unpack,
                               cudaStream_t st);
cudaError_t launch_pack_gauge(int prec, bool c12, const Geom& g, const double* canon, void* Ueven, void* Uodd,
                              cudaStream_t st);
cudaError_t launch_convert(int psrc, int pdst, const void* src, void* dst, long nsites, int Ls, const double* scale_dev,
                           double scale, cudaStream_t st);
cudaError_t launch_mooee(int prec, const void* in, void* out, long nsites, int Ls, bool dag, bool inverse, double d5,
                         double mass, double inv_d5, double inv_den, cudaStream_t st);
// Reductions over nsites site blocks. inner: a^+ b (complex); otherwise |a|^2. The result goes
// to scal[] according to kind.
cudaError_t launch_reduce(int prec, const void* a, const void* b, long nsites, int Ls, double* partials, double* scal,
                          int kind, int dst, cudaStream_t st);
// CG updates. xr: x += alpha p, r -= alpha Ap, |r|^2 -> finalised as FIN_BETA.
cudaError_t launch_cg_xr(int px, int pp, void* x, void* r, const void* p, const void* Ap, long nsites, int Ls,
                         double* partials, double* scal, cudaStream_t st);
// p = r + beta p.
// r -= alpha Ap and |r|^2 (finalised as FIN_BETA); x += alpha p, then (update_p) p = r + beta p.
cudaError_t launch_cg_r(int px, int pp, void* r, const void* Ap, long nsites, int Ls, double* partials, double* scal,
                        cudaStream_t st);
cudaError_t launch_cg_xp(int px, int pp, void* x, const void* r, void* p, long nsites, int Ls, const double* scal,
                         bool update_p, cudaStream_t st);
cudaError_t launch_cg_p(int px, int pp, const void* r, void* p, long nsites, int Ls, const double* scal,
                        cudaStream_t st);
// r = b - Ax (FP64) and |r|^2 -> scal[dst].
cudaError_t launch_residual64(const void* b, const void* Ax, void* r, long nsites, int Ls, double* partials,
                              double* scal, int dst, cudaStream_t st);
// x (FP64) += c * y (precision py), then y = 0, with c = *c_dev.
cudaError_t launch_accum_zero(int py, void* x, void* y, long nsites, int Ls, const double* c_dev, cudaStream_t st);
// y = a x + b y elementwise in precision p (a, b host scalars).
cudaError_t launch_axpby(int p, double a, const void* x, double b, void* y, long nsites, int Ls, cudaStream_t st);

}  // namespace gdwf
