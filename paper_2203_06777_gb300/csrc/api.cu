// C ABI of the domain-wall operator library (declared in include/grid_dwf.h): the operator
// handle, argument checking, the fused kernel sequences of M, Mpc and Mpc^+ Mpc, and the plain
// and mixed-precision CG solvers, driven from the host on the handle's stream.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/grid_dwf.h"
#include "dhop_ff.cuh"
#include "site_ops.cuh"

namespace gdwf {
cudaError_t launch_face_project(int prec, bool dag, const Geom& g, int plane, const void* in, float ph_first,
                                float ph_last, void* send_first, void* send_last, cudaStream_t st);
cudaError_t launch_force(int prec, bool c12, const Geom& g, const void* psi, const void* chi, const void* Ue,
                         const void* Uo, double* F, double* G, double coef, bool float_float, cudaStream_t st);
}

using namespace gdwf;

struct grid_dwf {
  Geom g;
  int Ls = 0;
  double M5 = 0, mass = 0;
  bool c12 = false;
  double d5 = 0, inv_d5 = 0, inv_den = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  size_t l2_bytes = (size_t)126 << 20;  // the device's L2 (read at create)
  double* U_canon = nullptr;            // canonical FP64 links, device
  void* gauge[4][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
  std::map<int, std::pair<void*, size_t>> ws;  // workspace buffers by id
  double* partials = nullptr;           // reduction partial sums
  double* scal = nullptr;               // CG scalars (device)
  double* host_scal = nullptr;          // pinned mirror of scal
  // CG: |r|^2 of each inner iteration copied to a pinned ring with an event, so that the host
  // reads an iteration's residual while the next iteration is already queued
  static constexpr int RING = 4;
  double* host_ring = nullptr;
  cudaEvent_t ring_ev[RING] = {};
  std::string err;
  bool sync_debug = false;
  // walk of the packed hopping launches in z-blocks of this many planes (-1: automatic; the
  // environment variable GRID_DWF_ZBLOCK, read at create, overrides it; 0 = lexicographic)
  int zblk = -1;
  // CG: the inner iteration whose residual decides a reliable update, counted back from the
  // current one (-1: automatic; GRID_DWF_CG_LAG, read at create, overrides it)
  int cg_lag = -1;
  // CG: the reliable-update threshold (the sloppy residual's drop since the last update); 0:
  // automatic (GRID_DWF_CG_DELTA, read at create, overrides it)
  double cg_delta = 0;
  // launch the packed hopping kernels as programmatic dependents of the previous kernel: the next
  // launch's CTAs become resident while the previous kernel's last CTAs run, and wait (before
  // their first load) for it to finish; 16^4 x 16 FP32 59.0 -> 56.3 us, FP16 41.1 -> 39.1 us per
  // full-lattice launch, bit-identical results (GRID_DWF_PDL=0, read at create, turns it off)
  int pdl = 1;
  // sites per CTA of the packed hopping kernels if smaller than the 128-thread default (0: the
  // default; GRID_DWF_SITES_PER_CTA, read at create, sets it)
  int spc = 0;
  int fp64_arith = GRID_DWF_FP64_ARITH_NATIVE;  // arithmetic of the FP64 hopping term
};

namespace {

// An NVTX range around each compute entry point, named after it, so that a timeline tool
// (nsys) shows the ABI calls over their kernels; a no-op when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

enum WsId : int {
  WS_TMP_E = 0,
  WS_TMP_O,
  WS_TMP_E2,
  WS_CHI,
  WS_CG_TE,
  WS_CG_BP,
  WS_CG_RHS,
  WS_CG_R,
  WS_CG_P,
  WS_CG_AP,
  WS_CG_TO,
  WS_CG_RS,
  WS_CG_XS,
  WS_CG_PS,
  WS_CG_APS,
  WS_CG_TOS,
  WS_CG_TES,
  WS_CANON_TMP,
  WS_PF_A,
  WS_PF_B,
  WS_PF_A32,
  WS_PF_B32,
  WS_CG_RED,
};

// Optional CG epilogue of a packed hop (see dhop_kernel.cuh): per-CTA partial sums
// into red; with r, the update r -= (*coef) * result instead of a stored result.
struct CgEpilogue {
  double* red = nullptr;
  float* r = nullptr;
  const double* coef = nullptr;
};

// Optional site range of a packed half-lattice hop (sites site_base .. site_base + nsites - 1) and,
// for the face planes of a block of a lattice split in t, the received faces and links.
struct HopRegion {
  int site_base = 0;
  int nsites = 0;
  const void* halo_fwd = nullptr;
  const void* halo_bwd = nullptr;
  const void* halo_links = nullptr;
};

int fail(grid_dwf_t* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int cuda_fail(grid_dwf_t* h, cudaError_t e, const char* where) {
  return fail(h, e == cudaErrorMemoryAllocation ? GRID_DWF_ERR_OOM : GRID_DWF_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(expr, where)                              \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

#define RET(expr)              \
  do {                         \
    int r_ = (expr);           \
    if (r_ != GRID_DWF_OK) return r_; \
  } while (0)

bool valid_prec(int p) { return p >= GRID_DWF_FP64 && p <= GRID_DWF_BF16; }

// A half field: V/2 site blocks of the padded Ls x 24 reals.
size_t half_bytes(const grid_dwf_t* h, int prec) {
  return (size_t)h->g.N4h * ls_padded(h->Ls) * 24 * prec_bytes(prec);
}

size_t subset_bytes(const grid_dwf_t* h, int prec, int subset) {
  return half_bytes(h, prec) * (subset == GRID_DWF_FULL ? 2 : 1);
}

int check_ptr(grid_dwf_t* h, const void* p, const char* name) {
  if (!p) return fail(h, GRID_DWF_ERR_INVALID_ARG, std::string(name) + " is null");
  if (reinterpret_cast<uintptr_t>(p) % 16) return fail(h, GRID_DWF_ERR_INVALID_ARG, std::string(name) + " is not 16-byte aligned");
  return GRID_DWF_OK;
}

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + nb && y < x + na;
}

int ws_get(grid_dwf_t* h, int id, size_t bytes, void** out) {
  auto it = h->ws.find(id);
  if (it != h->ws.end() && it->second.second >= bytes) {
    *out = it->second.first;
    return GRID_DWF_OK;
  }
  if (it != h->ws.end()) {
    cudaFree(it->second.first);
    h->ws.erase(it);
  }
  void* p = nullptr;
  CK(cudaMalloc(&p, bytes), "workspace allocation");
  h->ws[id] = {p, bytes};
  *out = p;
  return GRID_DWF_OK;
}

int finish(grid_dwf_t* h, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, where);
  if (h->sync_debug) {
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, where);
  }
  return GRID_DWF_OK;
}

int ensure_gauge(grid_dwf_t* h, int prec) {
  if (!h->U_canon) return fail(h, GRID_DWF_ERR_NO_GAUGE, "no gauge field set (call grid_dwf_set_gauge)");
  if (h->gauge[prec][0]) return GRID_DWF_OK;
  const size_t lb = link_bytes(prec_bytes(prec), h->c12);
  const size_t bytes = (size_t)h->g.N4h * 4 * lb;
  for (int p = 0; p < 2; ++p) CK(cudaMalloc(&h->gauge[prec][p], bytes), "gauge allocation");
  CK(launch_pack_gauge(prec, h->c12, h->g, h->U_canon, h->gauge[prec][0], h->gauge[prec][1], h->stream), "pack gauge");
  return GRID_DWF_OK;
}

// Whole sites per CTA of a hopping launch: as many as fill 128 threads (one per slice pair, or per
// slice in FP64), at most the half lattice; the packed kernels take fewer if the handle says so.
// Packed kernels: 8 sites (64 threads) for 8 slice pairs: measured at Ls = 16, 16 -> 8 sites per
// CTA (same warps per SM, a finer last wave) took the FP32 hop from 56.4 to 55.9 us at 16^4 and
// from 842 to 822 us at 32^4, FP16 from 589 to 580 us at 32^4, bit-identical. Otherwise, where
// one exists, the largest CTA of whole warps made of whole 4-site blocks: for 6 slice pairs
// (Ls = 11-12) 16 sites (96 threads) instead of 21 (126) took the full-lattice FP32 hop at
// 24^4 x 12 from 249 to 229 us, FP16 from 185 to 175 us, BF16 from 193 to 185 us (20 sites,
// 120 threads: 244 / 189 / 197 us).
int hop_sites_per_cta(const grid_dwf_t* h, int prec) {
  int spc = 128 / dhop_threads_per_site(prec, h->Ls);
  if (prec != GRID_DWF_FP64) {
    const int Lsh = ls_half(h->Ls);
    if (Lsh == 8) {
      spc = 8;
    } else {
      for (int s = spc - spc % 4; s >= 4; s -= 4)
        if ((s * Lsh) % 32 == 0) {
          spc = s;
          break;
        }
    }
  }
  if (prec != GRID_DWF_FP64 && h->spc > 0 && h->spc < spc) spc = h->spc;
  if (spc < 1) spc = 1;
  if (spc > h->g.N4h) spc = h->g.N4h;  // tiny lattices: one full CTA
  return spc;
}

// One half-lattice hopping application with its fused epilogue.
int dhop_half(grid_dwf_t* h, int prec, const void* in, void* out, int out_parity, bool dag, int pre, int post,
              double alpha, double beta, const void* aux, const void* in2 = nullptr, void* out2 = nullptr,
              const void* aux2 = nullptr, const CgEpilogue& epi = CgEpilogue(),
              const HopRegion& region = HopRegion()) {
  RET(ensure_gauge(h, prec));
  DhopArgs a;
  a.halo_fwd = region.halo_fwd;
  a.halo_bwd = region.halo_bwd;
  a.halo_links = region.halo_links;
  a.plane = h->g.Lxh * h->g.L[1] * h->g.L[2];
  a.region_sites = region.nsites;
  a.red = epi.red;
  a.r = epi.r;
  a.axpy_coef = epi.coef;
  a.red_base = 0;
  a.own_from = 0;
  a.pdl = h->pdl;
  a.in2 = in2;
  a.out2 = out2;
  a.aux2 = aux2;
  a.blocks1 = 0;
  a.in = in;
  a.out = out;
  a.aux = aux;
  a.Uout = h->gauge[prec][out_parity];
  a.Uin = h->gauge[prec][1 - out_parity];
  a.g = h->g;
  a.out_parity = out_parity;
  a.nsg = dhop_threads_per_site(prec, h->Ls);
  a.sites_per_cta = hop_sites_per_cta(h, prec);
  a.pre = pre;
  a.post = post;
  a.site_base = region.site_base;
  a.zblk = 0;
  a.ctas_per_plane = 1;
  a.interleave = 0;
  {
    // Automatic choice: an input t-plane is read again by the output planes t - 1 and t + 1, after
    // about two t-planes of input, output and links have passed through L2. The FP32 kernel walks
    // blocks of 8 (x, y) planes in z when that window exceeds half of L2 (32^4 x 16: 120 MB;
    // lexicographic walk 988 us, z-blocks of 2 / 4 / 8 / 16 planes 920 / 859 / 833 / 868 us) and
    // lexicographically otherwise (24^4 x 12: 40 MB, full-lattice hop 229 us against 240 us in
    // z-blocks of 8; 16^4 x 16: no change). The 16-bit kernels, bound by their arithmetic, gain
    // nothing.
    const int plane = h->g.Lxh * h->g.L[1];
    const size_t tplane = (size_t)plane * h->g.L[2];
    int zb = h->zblk;
    if (zb < 0) {
      const size_t window = 2 * tplane * ((size_t)ls_half(h->Ls) * 2 * 2 * 24 * 4 + 8 * 18 * 4);
      zb = (prec == GRID_DWF_FP32 && window > h->l2_bytes / 2) ? 8 : 0;
    }
    // FP32: both halves of a full-lattice launch in alternating CTAs when the reuse windows of both
    // fit in half of L2 together (the halves then share their link reads there): 16^4 x 16 55.3 ->
    // 54.2 us; where they do not fit it costs 4-8% (24^4 x 12 227 -> 236 us, 32^4 x 16 817 ->
    // 862 us, FP16 at 32^4 586 -> 634 us), and FP16 / BF16 at 16^4 gain nothing, so it is chosen
    // for FP32 below that size only.
    const size_t window_p = 2 * tplane * ((size_t)ls_half(h->Ls) * 2 * 2 * 24 * 4 + 8 * 18 * 4);
    a.interleave = (prec == GRID_DWF_FP32 && in2 != nullptr && 2 * window_p <= h->l2_bytes / 2) ? 1 : 0;
    if (prec != GRID_DWF_FP64 && region.nsites == 0 && zb > 0 && zb < h->g.L[2] && h->g.L[2] % zb == 0 &&
        plane % a.sites_per_cta == 0) {
      a.zblk = zb;
      a.ctas_per_plane = plane / a.sites_per_cta;
      a.div_cpp = make_fastdiv((uint32_t)a.ctas_per_plane);
      a.div_zblk = make_fastdiv((uint32_t)zb);
      a.div_lt = make_fastdiv((uint32_t)h->g.L[3]);
    }
  }
  a.alpha = alpha;
  a.beta = beta;
  a.d5 = h->d5;
  a.mass = h->mass;
  a.inv_d5 = h->inv_d5;
  a.inv_den = h->inv_den;
  int threads = a.nsg * a.sites_per_cta;
  int blocks = (h->g.N4h + a.sites_per_cta - 1) / a.sites_per_cta;
  const size_t rbytes = prec == GRID_DWF_FP64 ? 8 : 4;
  size_t smem = dhop_link_smem_bytes(prec, a.sites_per_cta, h->c12) +
                (post == POST_NONE                ? 0
                 : prec == GRID_DWF_FP64 ? (size_t)a.sites_per_cta * h->Ls * INV_SLICE_STRIDE * rbytes
                                         : (size_t)a.sites_per_cta * inv_site_stride(h->Ls) * rbytes);
  cudaError_t e;
  if (prec == GRID_DWF_FP64 && h->fp64_arith == GRID_DWF_FP64_ARITH_FLOAT_FLOAT) {
    smem = dhop_ff_smem_bytes(a.sites_per_cta, h->Ls, post != POST_NONE);
    e = launch_dhop_ff(a, dag, h->c12, threads, blocks, smem, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "dhop launch (float-float)");
    return GRID_DWF_OK;
  }
  switch (prec) {
    case GRID_DWF_FP64: e = launch_dhop<P64>(a, dag, h->c12, threads, blocks, smem, h->stream); break;
    case GRID_DWF_FP32: e = launch_dhop<P32>(a, dag, h->c12, threads, blocks, smem, h->stream); break;
    case GRID_DWF_FP16: e = launch_dhop<P16>(a, dag, h->c12, threads, blocks, smem, h->stream); break;
    default: e = launch_dhop<PB16>(a, dag, h->c12, threads, blocks, smem, h->stream); break;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "dhop launch");
  return GRID_DWF_OK;
}

// Both halves of a full-lattice hop (each output half from the other input half, independent):
// one launch for the packed precisions (one ramp-up and tail instead of two), two for FP64.
int dhop_full(grid_dwf_t* h, int prec, const char* in, char* out, bool dag, int pre, double alpha, double beta,
              const char* aux, const CgEpilogue& epi = CgEpilogue()) {
  const size_t hb = half_bytes(h, prec);
  if (prec == GRID_DWF_FP64) {
    RET(dhop_half(h, prec, in + hb, out, 0, dag, pre, POST_NONE, alpha, beta, aux));
    return dhop_half(h, prec, in, out + hb, 1, dag, pre, POST_NONE, alpha, beta, aux ? aux + hb : nullptr);
  }
  return dhop_half(h, prec, in + hb, out, 0, dag, pre, POST_NONE, alpha, beta, aux, in, out + hb,
                   aux ? aux + hb : nullptr, epi);
}

// Partial sums of a packed full-lattice launch with the norm epilogue: one per full CTA of
// either half, and one per half for the end CTAs of a ragged lattice.
int full_partials(const grid_dwf_t* h, int prec) {
  const int spc = hop_sites_per_cta(h, prec);
  const long N = h->g.N4h;
  return (int)(2 * (N / spc) + (N % spc ? 2 : 0));
}

// out_o = Mpc in_o (dag: Mpc^+), via t_e = Mooee^-1 D_eo in and out = Mooee in - D_oe t_e / 4.
int mpc_impl(grid_dwf_t* h, int prec, const void* in, void* out, bool dag, void* te) {
  RET(dhop_half(h, prec, in, te, 0, dag, PRE_NONE, dag ? POST_INV_DAG : POST_INV, 1.0, 0.0, nullptr));
  RET(dhop_half(h, prec, te, out, 1, dag, dag ? PRE_MOOEE_DAG : PRE_MOOEE, POST_NONE, -0.25, 1.0, in));
  return GRID_DWF_OK;
}

int mdagm_impl(grid_dwf_t* h, int prec, const void* in, void* out, void* to, void* te) {
  RET(mpc_impl(h, prec, in, to, false, te));
  RET(mpc_impl(h, prec, to, out, true, te));
  return GRID_DWF_OK;
}

int read_scalars(grid_dwf_t* h) {
  CK(cudaMemcpyAsync(h->host_scal, h->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, h->stream), "scalar read");
  CK(cudaStreamSynchronize(h->stream), "scalar read");
  return GRID_DWF_OK;
}

int write_scalar(grid_dwf_t* h, int idx, double v) {
  // staged through a pinned slot past the mirror so that the stream-ordered copy reads a stable value
  h->host_scal[S_COUNT + idx] = v;
  CK(cudaMemcpyAsync(h->scal + idx, h->host_scal + S_COUNT + idx, sizeof(double), cudaMemcpyHostToDevice, h->stream),
     "scalar write");
  return GRID_DWF_OK;
}

bool is_finite(double v) { return std::isfinite(v); }

}  // namespace

extern "C" {

const char* grid_dwf_status_string(int code) {
  switch (code) {
    case GRID_DWF_OK: return "ok";
    case GRID_DWF_ERR_INVALID_ARG: return "invalid argument";
    case GRID_DWF_ERR_CUDA: return "CUDA error";
    case GRID_DWF_ERR_OOM: return "out of device memory";
    case GRID_DWF_ERR_NOT_CONVERGED: return "solver did not converge";
    case GRID_DWF_ERR_NONFINITE: return "non-finite value";
    case GRID_DWF_ERR_ALIAS: return "output overlaps an input";
    case GRID_DWF_ERR_NO_GAUGE: return "no gauge field set";
    default: return "unknown status";
  }
}

const char* grid_dwf_last_error(const grid_dwf_t* h) { return h ? h->err.c_str() : "null handle"; }

int grid_dwf_create(const int dims[4], int Ls, double M5, double mass, const int bc[4], int compress12, void* stream,
                    grid_dwf_t** out) {
  if (!out || !dims) return GRID_DWF_ERR_INVALID_ARG;
  *out = nullptr;
  long V = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 2 || dims[m] % 2) return GRID_DWF_ERR_INVALID_ARG;
    V *= dims[m];
  }
  if (Ls < 1 || Ls > 128) return GRID_DWF_ERR_INVALID_ARG;  // FP64: one thread per slice, 128 per CTA
  if ((V / 2) * 8 >= (1L << 31)) return GRID_DWF_ERR_INVALID_ARG;
  if (!std::isfinite(M5) || !std::isfinite(mass)) return GRID_DWF_ERR_INVALID_ARG;
  const int defbc[4] = {1, 1, 1, -1};
  const int* b = bc ? bc : defbc;
  for (int m = 0; m < 4; ++m)
    if (b[m] != 1 && b[m] != -1) return GRID_DWF_ERR_INVALID_ARG;
  const double d5 = 5.0 - M5;
  if (d5 == 0.0) return GRID_DWF_ERR_INVALID_ARG;
  const double den = d5 + mass * std::pow(d5, -(double)(Ls - 1));
  // the fifth-dimension matrix has determinant d5^Ls + m per chirality
  if (den == 0.0 || !std::isfinite(1.0 / den) || std::pow(d5, (double)Ls) + mass == 0.0) return GRID_DWF_ERR_INVALID_ARG;

  grid_dwf_t* h = new grid_dwf_t();
  Geom& g = h->g;
  for (int m = 0; m < 4; ++m) {
    g.L[m] = dims[m];
    g.bc[m] = b[m];
  }
  g.Lxh = dims[0] / 2;
  g.Ls = Ls;
  g.N4h = (int)(V / 2);
  g.stride[0] = 1;
  g.stride[1] = g.Lxh;
  g.stride[2] = g.Lxh * dims[1];
  g.stride[3] = g.Lxh * dims[1] * dims[2];
  g.div_lxh = make_fastdiv(g.Lxh);
  g.div_ly = make_fastdiv(dims[1]);
  g.div_lz = make_fastdiv(dims[2]);
  h->Ls = Ls;
  h->M5 = M5;
  h->mass = mass;
  h->c12 = compress12 != 0;
  h->d5 = d5;
  h->inv_d5 = 1.0 / d5;
  h->inv_den = 1.0 / den;
  h->stream = static_cast<cudaStream_t>(stream);
  const char* sd = std::getenv("GRID_DWF_SYNC_DEBUG");
  h->sync_debug = sd && sd[0] == '1';
  const char* zbe = std::getenv("GRID_DWF_ZBLOCK");
  if (zbe) h->zblk = std::atoi(zbe);
  const char* spce = std::getenv("GRID_DWF_SITES_PER_CTA");
  if (spce) h->spc = std::atoi(spce);
  const char* pdle = std::getenv("GRID_DWF_PDL");
  if (pdle) h->pdl = std::atoi(pdle) != 0;
  const char* lge = std::getenv("GRID_DWF_CG_LAG");
  if (lge) h->cg_lag = std::atoi(lge) > 0 ? 1 : 0;
  const char* dle = std::getenv("GRID_DWF_CG_DELTA");
  if (dle) {
    const double d = std::atof(dle);
    if (d > 0 && d < 1) h->cg_delta = d;
  }
  cudaGetDevice(&h->device);
  {
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->device) == cudaSuccess && l2 > 0) h->l2_bytes = (size_t)l2;
  }
  cudaError_t e = cudaMalloc(&h->partials, sizeof(double) * 2 * RED_BLOCKS);
  if (e == cudaSuccess) e = cudaMalloc(&h->scal, sizeof(double) * S_COUNT);
  if (e == cudaSuccess) e = cudaMallocHost(&h->host_scal, sizeof(double) * (2 * S_COUNT + 1));
  if (e == cudaSuccess) e = cudaMallocHost(&h->host_ring, sizeof(double) * grid_dwf::RING);
  for (int k = 0; k < grid_dwf::RING && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&h->ring_ev[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemset(h->scal, 0, sizeof(double) * S_COUNT);
  if (e != cudaSuccess) {
    grid_dwf_destroy(h);
    return e == cudaErrorMemoryAllocation ? GRID_DWF_ERR_OOM : GRID_DWF_ERR_CUDA;
  }
  *out = h;
  return GRID_DWF_OK;
}

int grid_dwf_set_fp64_arith(grid_dwf_t* h, int mode) {
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (mode != GRID_DWF_FP64_ARITH_NATIVE && mode != GRID_DWF_FP64_ARITH_FLOAT_FLOAT)
    return fail(h, GRID_DWF_ERR_INVALID_ARG, "fp64 arithmetic mode must be NATIVE or FLOAT_FLOAT");
  h->fp64_arith = mode;
  return GRID_DWF_OK;
}

int grid_dwf_destroy(grid_dwf_t* h) {
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (h->stream) cudaStreamSynchronize(h->stream);
  cudaDeviceSynchronize();
  cudaFree(h->U_canon);
  for (auto& pp : h->gauge)
    for (auto& q : pp) cudaFree(q);
  for (auto& kv : h->ws) cudaFree(kv.second.first);
  cudaFree(h->partials);
  cudaFree(h->scal);
  cudaFreeHost(h->host_scal);
  cudaFreeHost(h->host_ring);
  for (auto& ev : h->ring_ev)
    if (ev) cudaEventDestroy(ev);
  delete h;
  return GRID_DWF_OK;
}

int grid_dwf_set_stream(grid_dwf_t* h, void* stream) {
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  h->stream = static_cast<cudaStream_t>(stream);
  return GRID_DWF_OK;
}

int grid_dwf_field_bytes(const grid_dwf_t* h, int precision, int subset, size_t* bytes) {
  if (!h || !bytes || !valid_prec(precision) || subset < 0 || subset > 2) return GRID_DWF_ERR_INVALID_ARG;
  *bytes = subset_bytes(h, precision, subset);
  return GRID_DWF_OK;
}

int grid_dwf_set_gauge(grid_dwf_t* h, const double* U) {
  const NvtxRange nvtx_("grid_dwf_set_gauge");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (!U) return fail(h, GRID_DWF_ERR_INVALID_ARG, "U is null");
  const size_t bytes = (size_t)h->g.N4h * 2 * 4 * 18 * sizeof(double);
  if (!h->U_canon) CK(cudaMalloc(&h->U_canon, bytes), "gauge allocation");
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, U);
  const bool on_device = e == cudaSuccess && (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
  cudaGetLastError();  // clear a possible error from querying an unregistered host pointer
  CK(cudaMemcpyAsync(h->U_canon, U, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream),
     "gauge copy");
  if (!on_device) CK(cudaStreamSynchronize(h->stream), "gauge copy");
  for (int p = 0; p < 4; ++p)
    if (h->gauge[p][0]) CK(launch_pack_gauge(p, h->c12, h->g, h->U_canon, h->gauge[p][0], h->gauge[p][1], h->stream), "pack gauge");
  return finish(h, "set_gauge");
}

int grid_dwf_pack(grid_dwf_t* h, int precision, int subset, const double* canonical, void* field) {
  const NvtxRange nvtx_("grid_dwf_pack");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (!valid_prec(precision) || subset < 0 || subset > 2) return fail(h, GRID_DWF_ERR_INVALID_ARG, "bad precision/subset");
  RET(check_ptr(h, canonical, "canonical"));
  RET(check_ptr(h, field, "field"));
  CK(launch_pack_spinor(precision, h->g, canonical, field, subset, false, h->stream), "pack");
  return finish(h, "pack");
}

int grid_dwf_unpack(grid_dwf_t* h, int precision, int subset, const void* field, double* canonical) {
  const NvtxRange nvtx_("grid_dwf_unpack");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (!valid_prec(precision) || subset < 0 || subset > 2) return fail(h, GRID_DWF_ERR_INVALID_ARG, "bad precision/subset");
  RET(check_ptr(h, canonical, "canonical"));
  RET(check_ptr(h, field, "field"));
  CK(launch_pack_spinor(precision, h->g, canonical, const_cast<void*>(field), subset, true, h->stream), "unpack");
  return finish(h, "unpack");
}

int grid_dwf_convert(grid_dwf_t* h, int src_precision, int dst_precision, int subset, const void* src, void* dst,
                     double scale) {
  const NvtxRange nvtx_("grid_dwf_convert");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (!valid_prec(src_precision) || !valid_prec(dst_precision) || subset < 0 || subset > 2)
    return fail(h, GRID_DWF_ERR_INVALID_ARG, "bad precision/subset");
  RET(check_ptr(h, src, "src"));
  RET(check_ptr(h, dst, "dst"));
  if (overlap(src, subset_bytes(h, src_precision, subset), dst, subset_bytes(h, dst_precision, subset)) &&
      !(src == dst && src_precision == dst_precision))
    return fail(h, GRID_DWF_ERR_ALIAS, "convert: dst overlaps src");
  const long nsites = (long)h->g.N4h * (subset == GRID_DWF_FULL ? 2 : 1);
  CK(launch_convert(src_precision, dst_precision, src, dst, nsites, h->Ls, nullptr, scale, h->stream), "convert");
  return finish(h, "convert");
}

int grid_dwf_dhop(grid_dwf_t* h, int precision, const void* in, void* out, int parity, int dag) {
  const NvtxRange nvtx_("grid_dwf_dhop");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (!valid_prec(precision) || parity < 0 || parity > 2) return fail(h, GRID_DWF_ERR_INVALID_ARG, "bad precision/parity");
  RET(check_ptr(h, in, "in"));
  RET(check_ptr(h, out, "out"));
  const int subset = parity == 2 ? GRID_DWF_FULL : GRID_DWF_EVEN;
  const size_t nb = subset_bytes(h, precision, subset);
  if (overlap(in, nb, out, nb)) return fail(h, GRID_DWF_ERR_ALIAS, "dhop: out overlaps in");
  if (parity == 2) {
    RET(dhop_full(h, precision, static_cast<const char*>(in), static_cast<char*>(out), dag != 0, PRE_NONE, 1.0, 0.0,
                  nullptr));
  } else {
    RET(dhop_half(h, precision, in, out, parity, dag != 0, PRE_NONE, POST_NONE, 1.0, 0.0, nullptr));
  }
  return finish(h, "dhop");
}

int grid_dwf_mooee(grid_dwf_t* h, int precision, int subset, const void* in, void* out, int dag, int inverse) {
  const NvtxRange nvtx_("grid_dwf_mooee");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (!valid_prec(precision) || subset < 0 || subset > 2) return fail(h, GRID_DWF_ERR_INVALID_ARG, "bad precision/subset");
  RET(check_ptr(h, in, "in"));
  RET(check_ptr(h, out, "out"));
  const size_t nb = subset_bytes(h, precision, subset);
  if (in != out && overlap(in, nb, out, nb)) return fail(h, GRID_DWF_ERR_ALIAS, "mooee: partial overlap");
  const long nsites = (long)h->g.N4h * (subset == GRID_DWF_FULL ? 2 : 1);
  CK(launch_mooee(precision, in, out, nsites, h->Ls, dag != 0, inverse != 0, h->d5, h->mass, h->inv_d5, h->inv_den,
                  h->stream),
     "mooee");
  return finish(h, "mooee");
}

int grid_dwf_m(grid_dwf_t* h, int precision, const void* in, void* out, int dag) {
  const NvtxRange nvtx_("grid_dwf_m");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (!valid_prec(precision)) return fail(h, GRID_DWF_ERR_INVALID_ARG, "bad precision");
  RET(check_ptr(h, in, "in"));
  RET(check_ptr(h, out, "out"));
  const size_t nb = subset_bytes(h, precision, GRID_DWF_FULL);
  if (overlap(in, nb, out, nb)) return fail(h, GRID_DWF_ERR_ALIAS, "m: out overlaps in");
  const char* ic = static_cast<const char*>(in);
  const int pre = dag ? PRE_MOOEE_DAG : PRE_MOOEE;
  RET(dhop_full(h, precision, ic, static_cast<char*>(out), dag != 0, pre, -0.5, 1.0, ic));
  return finish(h, "m");
}

int grid_dwf_mpc(grid_dwf_t* h, int precision, const void* in, void* out, int dag, void* tmp_even) {
  const NvtxRange nvtx_("grid_dwf_mpc");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (!valid_prec(precision)) return fail(h, GRID_DWF_ERR_INVALID_ARG, "bad precision");
  RET(check_ptr(h, in, "in"));
  RET(check_ptr(h, out, "out"));
  const size_t hb = half_bytes(h, precision);
  if (overlap(in, hb, out, hb)) return fail(h, GRID_DWF_ERR_ALIAS, "mpc: out overlaps in");
  void* te = tmp_even;
  if (!te) RET(ws_get(h, WS_TMP_E, hb, &te));
  RET(check_ptr(h, te, "tmp_even"));
  if (overlap(te, hb, in, hb) || overlap(te, hb, out, hb)) return fail(h, GRID_DWF_ERR_ALIAS, "mpc: tmp overlaps");
  RET(mpc_impl(h, precision, in, out, dag != 0, te));
  return finish(h, "mpc");
}

int grid_dwf_mdagm(grid_dwf_t* h, int precision, const void* in, void* out, void* tmp_odd, void* tmp_even) {
  const NvtxRange nvtx_("grid_dwf_mdagm");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (!valid_prec(precision)) return fail(h, GRID_DWF_ERR_INVALID_ARG, "bad precision");
  RET(check_ptr(h, in, "in"));
  RET(check_ptr(h, out, "out"));
  const size_t hb = half_bytes(h, precision);
  if (overlap(in, hb, out, hb)) return fail(h, GRID_DWF_ERR_ALIAS, "mdagm: out overlaps in");
  void* to = tmp_odd;
  void* te = tmp_even;
  if (!to) RET(ws_get(h, WS_TMP_O, hb, &to));
  if (!te) RET(ws_get(h, WS_TMP_E, hb, &te));
  RET(check_ptr(h, to, "tmp_odd"));
  RET(check_ptr(h, te, "tmp_even"));
  if (overlap(to, hb, in, hb) || overlap(to, hb, out, hb) || overlap(te, hb, in, hb) || overlap(te, hb, out, hb) ||
      overlap(to, hb, te, hb))
    return fail(h, GRID_DWF_ERR_ALIAS, "mdagm: scratch overlaps");
  RET(mdagm_impl(h, precision, in, out, to, te));
  return finish(h, "mdagm");
}

int grid_dwf_norm2(grid_dwf_t* h, int precision, int subset, const void* a, double* result) {
  const NvtxRange nvtx_("grid_dwf_norm2");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (!valid_prec(precision) || subset < 0 || subset > 2 || !result)
    return fail(h, GRID_DWF_ERR_INVALID_ARG, "bad precision/subset/result");
  RET(check_ptr(h, a, "a"));
  const long nsites = (long)h->g.N4h * (subset == GRID_DWF_FULL ? 2 : 1);
  CK(launch_reduce(precision, a, nullptr, nsites, h->Ls, h->partials, h->scal, FIN_STORE, S_TMP0, h->stream), "norm2");
  RET(read_scalars(h));
  *result = h->host_scal[S_TMP0];
  return GRID_DWF_OK;
}

int grid_dwf_inner(grid_dwf_t* h, int precision, int subset, const void* a, const void* b, double result[2]) {
  const NvtxRange nvtx_("grid_dwf_inner");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (!valid_prec(precision) || subset < 0 || subset > 2 || !result)
    return fail(h, GRID_DWF_ERR_INVALID_ARG, "bad precision/subset/result");
  RET(check_ptr(h, a, "a"));
  RET(check_ptr(h, b, "b"));
  const long nsites = (long)h->g.N4h * (subset == GRID_DWF_FULL ? 2 : 1);
  CK(launch_reduce(precision, a, b, nsites, h->Ls, h->partials, h->scal, FIN_STORE, S_TMP0, h->stream), "inner");
  RET(read_scalars(h));
  result[0] = h->host_scal[S_TMP0];
  result[1] = h->host_scal[S_TMP1];
  return GRID_DWF_OK;
}

}  // extern "C"

extern "C" {

// ---------------------------------------------------------------- blocks of a lattice split in t

namespace {
int halo_checks(grid_dwf_t* h, int precision) {
  if (precision != GRID_DWF_FP32 && precision != GRID_DWF_FP16 && precision != GRID_DWF_BF16)
    return fail(h, GRID_DWF_ERR_INVALID_ARG, "halo: FP32, FP16 or BF16 fields only");
  const int plane = h->g.Lxh * h->g.L[1] * h->g.L[2];
  if (plane % hop_sites_per_cta(h, precision) != 0)
    return fail(h, GRID_DWF_ERR_INVALID_ARG, "halo: a t-plane must hold whole CTAs of sites");
  return GRID_DWF_OK;
}
}  // namespace

int grid_dwf_face_bytes(const grid_dwf_t* h, int precision, size_t* face_bytes, size_t* link_face_bytes) {
  if (!h || !face_bytes || !link_face_bytes || !valid_prec(precision)) return GRID_DWF_ERR_INVALID_ARG;
  const size_t plane = (size_t)h->g.Lxh * h->g.L[1] * h->g.L[2];
  *face_bytes = plane * ls_half(h->Ls) * 6 * 16;
  *link_face_bytes = plane * link_bytes(prec_bytes(precision), h->c12);
  return GRID_DWF_OK;
}

int grid_dwf_face_project(grid_dwf_t* h, int precision, const void* in, int dag, int phase_first, int phase_last,
                          void* send_first, void* send_last) {
  const NvtxRange nvtx_("grid_dwf_face_project");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  RET(halo_checks(h, precision));
  if ((phase_first != 1 && phase_first != -1) || (phase_last != 1 && phase_last != -1))
    return fail(h, GRID_DWF_ERR_INVALID_ARG, "face_project: phases must be +1 or -1");
  RET(check_ptr(h, in, "in"));
  RET(check_ptr(h, send_first, "send_first"));
  RET(check_ptr(h, send_last, "send_last"));
  const int plane = h->g.Lxh * h->g.L[1] * h->g.L[2];
  CK(launch_face_project(precision, dag != 0, h->g, plane, in, (float)phase_first, (float)phase_last, send_first,
                         send_last, h->stream),
     "face_project");
  return finish(h, "face_project");
}

int grid_dwf_face_links(grid_dwf_t* h, int precision, int out_parity, void* links_last) {
  const NvtxRange nvtx_("grid_dwf_face_links");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  RET(halo_checks(h, precision));
  if (out_parity != GRID_DWF_EVEN && out_parity != GRID_DWF_ODD)
    return fail(h, GRID_DWF_ERR_INVALID_ARG, "face_links: parity must be EVEN or ODD");
  RET(check_ptr(h, links_last, "links_last"));
  RET(ensure_gauge(h, precision));
  const size_t lb = link_bytes(prec_bytes(precision), h->c12);
  const int plane = h->g.Lxh * h->g.L[1] * h->g.L[2];
  const char* src = static_cast<const char*>(h->gauge[precision][1 - out_parity]) +
                    ((size_t)(h->g.N4h - plane) * 4 + 3) * lb;
  CK(cudaMemcpy2DAsync(links_last, lb, src, 4 * lb, lb, plane, cudaMemcpyDeviceToDevice, h->stream), "face_links");
  return finish(h, "face_links");
}

int grid_dwf_dhop_region(grid_dwf_t* h, int precision, const void* in, void* out, int out_parity, int dag,
                         int region, const void* recv_fwd, const void* recv_bwd, const void* links_bwd) {
  const NvtxRange nvtx_("grid_dwf_dhop_region");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  RET(halo_checks(h, precision));
  if (out_parity != GRID_DWF_EVEN && out_parity != GRID_DWF_ODD)
    return fail(h, GRID_DWF_ERR_INVALID_ARG, "dhop_region: parity must be EVEN or ODD");
  if (region != GRID_DWF_REGION_INTERIOR && region != GRID_DWF_REGION_FACES)
    return fail(h, GRID_DWF_ERR_INVALID_ARG, "dhop_region: region must be INTERIOR or FACES");
  RET(check_ptr(h, in, "in"));
  RET(check_ptr(h, out, "out"));
  const size_t nb = half_bytes(h, precision);
  if (overlap(in, nb, out, nb)) return fail(h, GRID_DWF_ERR_ALIAS, "dhop_region: out overlaps in");
  const int plane = h->g.Lxh * h->g.L[1] * h->g.L[2];
  if (region == GRID_DWF_REGION_INTERIOR) {
    if (h->g.N4h > 2 * plane) {  // Lt >= 3
      HopRegion r;
      r.site_base = plane;
      r.nsites = h->g.N4h - 2 * plane;
      RET(dhop_half(h, precision, in, out, out_parity, dag != 0, PRE_NONE, POST_NONE, 1.0, 0.0, nullptr, nullptr,
                    nullptr, nullptr, CgEpilogue(), r));
    }
    return finish(h, "dhop_region");
  }
  RET(check_ptr(h, recv_fwd, "recv_fwd"));
  RET(check_ptr(h, recv_bwd, "recv_bwd"));
  RET(check_ptr(h, links_bwd, "links_bwd"));
  for (int k = 0; k < 2; ++k) {  // the first t-plane, then the last
    HopRegion r;
    r.site_base = k == 0 ? 0 : h->g.N4h - plane;
    r.nsites = plane;
    r.halo_fwd = recv_fwd;
    r.halo_bwd = recv_bwd;
    r.halo_links = links_bwd;
    RET(dhop_half(h, precision, in, out, out_parity, dag != 0, PRE_NONE, POST_NONE, 1.0, 0.0, nullptr, nullptr,
                  nullptr, nullptr, CgEpilogue(), r));
  }
  return finish(h, "dhop_region");
}

}  // extern "C"

namespace {

struct CgResult {
  int iters = 0;
  int updates = 0;
  bool converged = false;
  double true_res = 0;
  double flops = 0;
};

// Solve Mpc^+ Mpc x_o = rhs for odd half fields in FP64 device layout, from the initial guess in
// x_o, by plain FP64 CG or by FP64 defect correction around an inner CG in a lower storage
// precision with reliable updates (mode). rhs is only read. Stops when the FP64 true residual
// |rhs - Mpc^+ Mpc x_o| / |rhs| is at most tol, or after maxiter iterations; the true residual
// is recomputed in FP64 at the end either way and returned with the counts.
int cg_normal(grid_dwf_t* h, const void* rhs, void* xo_, double tol, int maxiter, int mode, CgResult& res) {
  const size_t hb = half_bytes(h, GRID_DWF_FP64);
  const long N = h->g.N4h;
  const int Ls = h->Ls;
  const double half_flops = 1320.0 * (double)N * Ls;
  double flops = 0;
  char* xo = static_cast<char*>(xo_);
  void *te, *r, *p, *Ap, *to;
  RET(ws_get(h, WS_CG_TE, hb, &te));
  RET(ws_get(h, WS_CG_R, hb, &r));
  RET(ws_get(h, WS_CG_AP, hb, &Ap));
  RET(ws_get(h, WS_CG_TO, hb, &to));
  const int P = GRID_DWF_FP64;
  CK(launch_reduce(P, rhs, nullptr, N, Ls, h->partials, h->scal, FIN_STORE, S_TMP1, h->stream), "cg norm");
  CK(launch_reduce(P, xo, nullptr, N, Ls, h->partials, h->scal, FIN_STORE, S_TMP0, h->stream), "cg guess norm");
  RET(read_scalars(h));
  const double rhs_norm = std::sqrt(h->host_scal[S_TMP1]);
  double rr;
  if (h->host_scal[S_TMP0] == 0.0) {
    // zero initial guess: r = rhs exactly, no FP64 Mpc^+ Mpc needed
    CK(launch_convert(P, P, rhs, r, N, Ls, nullptr, 1.0, h->stream), "cg residual");
    rr = h->host_scal[S_TMP1];
    RET(write_scalar(h, S_RR, rr));
  } else {
    // true residual r = rhs - A x_o
    RET(mdagm_impl(h, P, xo, Ap, to, te));
    flops += 4 * half_flops;
    CK(launch_residual64(rhs, Ap, r, N, Ls, h->partials, h->scal, S_RR, h->stream), "cg residual");
    RET(read_scalars(h));
    rr = h->host_scal[S_RR];
  }
  if (!is_finite(rr) || !is_finite(rhs_norm)) return fail(h, GRID_DWF_ERR_NONFINITE, "cg: non-finite source or guess");
  const double target = tol * rhs_norm;
  int iters = 0, updates = 0;
  bool converged = std::sqrt(rr) <= target;
  double true_res = rhs_norm > 0 ? std::sqrt(rr) / rhs_norm : 0.0;
  bool rr_is_true = true;  // rr is the FP64 true residual of the current x_o (no recomputation needed)

  if (mode == GRID_DWF_CG_FP64) {
    RET(ws_get(h, WS_CG_P, hb, &p));
    CK(launch_convert(P, P, r, p, N, Ls, nullptr, 1.0, h->stream), "cg init");
    RET(write_scalar(h, S_PSCALE, 1.0));
    while (!converged && iters < maxiter) {
      RET(mdagm_impl(h, P, p, Ap, to, te));
      CK(launch_reduce(P, p, Ap, N, Ls, h->partials, h->scal, FIN_ALPHA, 0, h->stream), "cg pAp");
      CK(launch_cg_xr(P, P, xo, r, p, Ap, N, Ls, h->partials, h->scal, h->stream), "cg update");
      CK(launch_cg_p(P, P, r, p, N, Ls, h->scal, h->stream), "cg p");
      flops += 4 * half_flops;
      ++iters;
      RET(read_scalars(h));
      rr = h->host_scal[S_RR];
      rr_is_true = false;  // the recursively updated residual
      if (!is_finite(rr)) return fail(h, GRID_DWF_ERR_NONFINITE, "cg: non-finite residual");
      converged = std::sqrt(rr) <= target;
    }
  } else {
    const int PS = mode == GRID_DWF_CG_MIXED_FP32 ? GRID_DWF_FP32 : mode == GRID_DWF_CG_MIXED_FP16 ? GRID_DWF_FP16 : GRID_DWF_BF16;
    const size_t hs32 = half_bytes(h, GRID_DWF_FP32), hss = half_bytes(h, PS);
    void *rs, *xs, *ps, *aps, *tos, *tes;
    RET(ws_get(h, WS_CG_RS, hs32, &rs));
    RET(ws_get(h, WS_CG_XS, hs32, &xs));
    RET(ws_get(h, WS_CG_PS, hss, &ps));
    RET(ws_get(h, WS_CG_APS, hss, &aps));
    RET(ws_get(h, WS_CG_TOS, hss, &tos));
    RET(ws_get(h, WS_CG_TES, hss, &tes));
    RET(ensure_gauge(h, PS));
    const double nreal = (double)N * Ls * 24;
    // Reliable update when the sloppy residual has dropped by delta since the last one. FP32
    // inner solves keep their recursion accurate over four decades; with 16-bit storage the
    // recursion drifts sooner (a smaller delta there adds iterations or stalls). Measured to a
    // 1e-10 true residual: FP32 at 24^4 x 12, delta 1e-3 / 1e-4 / 1e-5: 4 / 3 / 3 FP64 Mpc^+ Mpc
    // recomputations in 170 / 170 / 172 iterations, 0.235 / 0.220 / 0.222 s; at 32^4 x 16 (m =
    // 0.005) 4 / 3 / 4 in 228 / 230 / 241 iterations, 1.013 / 0.961 / 1.054 s. FP16 at 24^4 x 12,
    // delta 0.1 / 0.03 / 0.01 / 3e-3: 170 / 171 / 171 / 283 iterations, and at 1e-3 742; BF16 at
    // 0.1 / 0.03 / 0.01: 197 / 223 / 381, and no convergence at 3e-3.
    const double delta = h->cg_delta > 0 ? h->cg_delta : PS == GRID_DWF_FP32 ? 1e-4 : 0.03;
    double sigma = std::sqrt(nreal) / std::sqrt(rr);
    CK(launch_convert(P, GRID_DWF_FP32, r, rs, N, Ls, nullptr, sigma, h->stream), "cg init");
    CK(launch_convert(GRID_DWF_FP32, PS, rs, ps, N, Ls, nullptr, 1.0, h->stream), "cg init");
    CK(cudaMemsetAsync(xs, 0, hs32, h->stream), "cg init");
    CK(launch_reduce(GRID_DWF_FP32, rs, nullptr, N, Ls, h->partials, h->scal, FIN_STORE, S_RR, h->stream), "cg init");
    RET(write_scalar(h, S_PSCALE, 1.0));
    RET(read_scalars(h));
    double rr_s = h->host_scal[S_RR];
    double rr_max = rr_s;
    // The normal operator's launches with the vector algebra fused (18-real links): p^+ A p is
    // |Mpc p|^2, summed in the epilogue of Mpc's second launch, and r -= alpha A p happens in the
    // epilogue of Mpc^+'s second launch, so A p is never stored. Partial sums: one per CTA.
    // Both use the FP32 results before they are rounded to the storage format.
    const bool fused = !h->c12;
    double* red = nullptr;
    int nred = 0;
    if (fused) {
      const int spc = hop_sites_per_cta(h, PS);
      nred = (int)(N / spc) + (N % spc ? 1 : 0);  // the full CTAs, and the end CTA if there is one
      void* rp = nullptr;
      RET(ws_get(h, WS_CG_RED, sizeof(double) * (size_t)nred, &rp));
      red = static_cast<double*>(rp);
    }
    int last_update = 0;  // iteration of the last reliable update (its |r|^2 is on another scale)
    // The decision reads the previous iteration's residual (the GPU never waits for the host)
    // except with BF16 storage, whose 8-bit recursion drifts fast enough that one iteration's
    // delay before each reliable update cost it 309 iterations instead of 225 at 24^4 x 12 (FP32:
    // 170 / 169 at the same time; FP16: 171 / 169, and 0.230 s against 0.244 s).
    const int lag = h->cg_lag >= 0 ? h->cg_lag : (PS == GRID_DWF_BF16 ? 0 : 1);
    while (!converged && iters < maxiter) {
      if (fused) {
        CgEpilogue norm;
        norm.red = red;
        CgEpilogue axpy;
        axpy.red = red;
        axpy.r = static_cast<float*>(rs);
        axpy.coef = h->scal + S_ALPHA;
        RET(dhop_half(h, PS, ps, tes, 0, false, PRE_NONE, POST_INV, 1.0, 0.0, nullptr));
        RET(dhop_half(h, PS, tes, tos, 1, false, PRE_MOOEE, POST_NONE, -0.25, 1.0, ps, nullptr, nullptr, nullptr, norm));
        CK(launch_finalize_n(red, nred, h->scal, FIN_ALPHA, 0, h->stream), "cg pAp");
        RET(dhop_half(h, PS, tos, tes, 0, true, PRE_NONE, POST_INV_DAG, 1.0, 0.0, nullptr));
        RET(dhop_half(h, PS, tes, aps, 1, true, PRE_MOOEE_DAG, POST_NONE, -0.25, 1.0, tos, nullptr, nullptr, nullptr,
                      axpy));
        CK(launch_finalize_n(red, nred, h->scal, FIN_BETA, 0, h->stream), "cg update");
      } else {
        RET(mdagm_impl(h, PS, ps, aps, tos, tes));
        CK(launch_reduce(PS, ps, aps, N, Ls, h->partials, h->scal, FIN_ALPHA, 0, h->stream), "cg pAp");
        // r -= alpha Ap now; x += alpha p is deferred to the pass that updates p (one read of p)
        CK(launch_cg_r(GRID_DWF_FP32, PS, rs, aps, N, Ls, h->partials, h->scal, h->stream), "cg update");
      }
      flops += 4 * half_flops;
      ++iters;
      rr_is_true = false;  // x_s has moved since the last true residual
      // |r|^2 of this iteration to the host ring; the decision below reads the previous
      // iteration's, which is complete or nearly so while this one is still queued
      const int slot = iters % grid_dwf::RING;
      CK(cudaMemcpyAsync(h->host_ring + slot, h->scal + S_RRNEW, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
         "cg residual copy");
      CK(cudaEventRecord(h->ring_ev[slot], h->stream), "cg residual copy");
      bool reliable = iters == maxiter;
      if (iters - lag > last_update) {
        const int prev = (iters - lag) % grid_dwf::RING;
        CK(cudaEventSynchronize(h->ring_ev[prev]), "cg residual read");
        const double rp = h->host_ring[prev];
        if (!is_finite(rp)) return fail(h, GRID_DWF_ERR_NONFINITE, "cg: non-finite sloppy residual");
        if (rp < delta * delta * rr_max || std::sqrt(rp) / sigma <= target) reliable = true;
      }
      if (reliable) {
        // reliable update (one iteration after the residual that called for it): complete x_s (the
        // pending alpha p), fold it into x, recompute the true residual in FP64, rescale
        RET(read_scalars(h));
        rr_s = h->host_scal[S_RRNEW];
        const double rr_old_s = h->host_scal[S_RROLD];  // |r_s|^2 before this step (the denominator of beta)
        if (!is_finite(rr_s)) return fail(h, GRID_DWF_ERR_NONFINITE, "cg: non-finite sloppy residual");
        CK(launch_cg_xp(GRID_DWF_FP32, PS, xs, rs, ps, N, Ls, h->scal, false, h->stream), "cg reliable");
        RET(write_scalar(h, S_TMP0, 1.0 / sigma));
        CK(launch_accum_zero(GRID_DWF_FP32, xo, xs, N, Ls, h->scal + S_TMP0, h->stream), "cg reliable");
        RET(mdagm_impl(h, P, xo, Ap, to, te));
        flops += 4 * half_flops;
        CK(launch_residual64(rhs, Ap, r, N, Ls, h->partials, h->scal, S_TMP1, h->stream), "cg reliable");
        RET(read_scalars(h));
        ++updates;
        last_update = iters;
        const double rr64 = h->host_scal[S_TMP1];
        if (!is_finite(rr64)) return fail(h, GRID_DWF_ERR_NONFINITE, "cg: non-finite true residual");
        rr = rr64;
        rr_is_true = true;  // x_s was folded into x_o and zeroed: rr64 is the residual of x_o
        if (std::sqrt(rr64) <= target) {
          converged = true;
          break;
        }
        const double sigma_new = std::sqrt(nreal) / std::sqrt(rr64);
        CK(launch_convert(P, GRID_DWF_FP32, r, rs, N, Ls, nullptr, sigma_new, h->stream), "cg reliable");
        CK(launch_reduce(GRID_DWF_FP32, rs, nullptr, N, Ls, h->partials, h->scal, FIN_STORE, S_RR, h->stream),
           "cg reliable");
        // beta (true units) = |r_true|^2 / |r_old|^2 with |r_old|^2 = rr_old_s / sigma^2; the stored
        // p carries scale sigma and must move to sigma_new.
        const double beta = rr64 * sigma * sigma / rr_old_s;
        RET(write_scalar(h, S_BETA, beta * sigma_new / sigma));
        RET(read_scalars(h));
        rr_s = h->host_scal[S_RR];
        rr_max = rr_s;
        sigma = sigma_new;
        rr = rr64;
        if (iters == maxiter) break;
        CK(launch_cg_p(GRID_DWF_FP32, PS, rs, ps, N, Ls, h->scal, h->stream), "cg p");  // x is complete: p alone
      } else {
        CK(launch_cg_xp(GRID_DWF_FP32, PS, xs, rs, ps, N, Ls, h->scal, true, h->stream), "cg xp");
      }
    }
  }
  // final true residual of the normal equations, FP64 (already known when the loop ended on a
  // reliable update or did not run)
  double rr_final = rr;
  if (!rr_is_true) {
    RET(mdagm_impl(h, P, xo, Ap, to, te));
    flops += 4 * half_flops;
    CK(launch_residual64(rhs, Ap, r, N, Ls, h->partials, h->scal, S_TMP0, h->stream), "cg final");
    RET(read_scalars(h));
    rr_final = h->host_scal[S_TMP0];
  }
  true_res = rhs_norm > 0 ? std::sqrt(rr_final) / rhs_norm : 0.0;
  res.iters = iters;
  res.updates = updates;
  res.true_res = true_res;
  res.converged = true_res <= tol;
  res.flops = flops;
  return GRID_DWF_OK;
}

}  // namespace

extern "C" {

int grid_dwf_cg(grid_dwf_t* h, const void* b, void* x, double tol, int maxiter, int mode, grid_dwf_cg_stats* stats) {
  const NvtxRange nvtx_("grid_dwf_cg");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (mode < GRID_DWF_CG_FP64 || mode > GRID_DWF_CG_MIXED_BF16 || !(tol > 0) || maxiter < 0)
    return fail(h, GRID_DWF_ERR_INVALID_ARG, "cg: bad mode/tol/maxiter");
  RET(check_ptr(h, b, "b"));
  RET(check_ptr(h, x, "x"));
  const size_t hb = half_bytes(h, GRID_DWF_FP64);
  if (overlap(b, 2 * hb, x, 2 * hb)) return fail(h, GRID_DWF_ERR_ALIAS, "cg: x overlaps b");
  const auto t0 = std::chrono::steady_clock::now();
  CK(cudaStreamSynchronize(h->stream), "cg start");
  const long N = h->g.N4h;
  const int Ls = h->Ls;
  const double half_flops = 1320.0 * (double)N * Ls;
  const char* be = static_cast<const char*>(b);
  const char* bo = be + hb;
  char* xe = static_cast<char*>(x);
  char* xo = xe + hb;
  void *te, *bp, *rhs;
  RET(ws_get(h, WS_CG_TE, hb, &te));
  RET(ws_get(h, WS_CG_BP, hb, &bp));
  RET(ws_get(h, WS_CG_RHS, hb, &rhs));
  const int P = GRID_DWF_FP64;
  // Schur source: b'_o = b_o + D_oe Mooee^-1 b_e / 2; rhs = Mpc^+ b'_o
  CK(launch_mooee(P, be, te, N, Ls, false, true, h->d5, h->mass, h->inv_d5, h->inv_den, h->stream), "cg source");
  RET(dhop_half(h, P, te, bp, 1, false, PRE_AUX, POST_NONE, 0.5, 1.0, bo));
  RET(mpc_impl(h, P, bp, rhs, true, te));
  CgResult res;
  RET(cg_normal(h, rhs, xo, tol, maxiter, mode, res));
  // x_e = Mooee^-1 (b_e + D_eo x_o / 2)
  RET(dhop_half(h, P, xo, xe, 0, false, PRE_AUX, POST_INV, 0.5, 1.0, be));
  CK(cudaStreamSynchronize(h->stream), "cg end");
  const auto t1 = std::chrono::steady_clock::now();
  if (stats) {
    stats->iterations = res.iters;
    stats->reliable_updates = res.updates;
    stats->converged = res.converged ? 1 : 0;
    stats->true_residual = res.true_res;
    stats->seconds = std::chrono::duration<double>(t1 - t0).count();
    stats->flops = res.flops + 4 * half_flops;
  }
  if (!res.converged) return fail(h, GRID_DWF_ERR_NOT_CONVERGED, "cg: tolerance not reached within maxiter");
  return finish(h, "cg");
}

int grid_dwf_force(grid_dwf_t* h, int precision, const void* psi, void* chi, double* F, double* G, double* S_out) {
  const NvtxRange nvtx_("grid_dwf_force");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (precision != GRID_DWF_FP64 && precision != GRID_DWF_FP32)
    return fail(h, GRID_DWF_ERR_INVALID_ARG, "force: precision must be FP64 or FP32");
  RET(check_ptr(h, psi, "psi"));
  const size_t fb = subset_bytes(h, precision, GRID_DWF_FULL);
  void* c = chi;
  if (!c) RET(ws_get(h, WS_CHI, fb, &c));
  RET(check_ptr(h, c, "chi"));
  if (overlap(psi, fb, c, fb)) return fail(h, GRID_DWF_ERR_ALIAS, "force: chi overlaps psi");
  const size_t gb = (size_t)h->g.N4h * 2 * 4 * 18 * sizeof(double);
  if (F && (overlap(F, gb, psi, fb) || overlap(F, gb, c, fb))) return fail(h, GRID_DWF_ERR_ALIAS, "force: F overlaps");
  if (G && (overlap(G, gb, psi, fb) || overlap(G, gb, c, fb))) return fail(h, GRID_DWF_ERR_ALIAS, "force: G overlaps");
  if (precision == GRID_DWF_FP32 && !h->c12) {
    // chi = M psi with |chi|^2 summed in the same launch (one partial per CTA, FP64 across CTAs)
    const int nred = full_partials(h, precision);
    void* rp = nullptr;
    RET(ws_get(h, WS_CG_RED, sizeof(double) * (size_t)nred, &rp));
    CgEpilogue norm;
    norm.red = static_cast<double*>(rp);
    const char* ic = static_cast<const char*>(psi);
    RET(dhop_full(h, precision, ic, static_cast<char*>(c), false, PRE_MOOEE, -0.5, 1.0, ic, norm));
    CK(launch_finalize_n(norm.red, nred, h->scal, FIN_STORE, S_TMP0, h->stream), "force action");
  } else {
    RET(grid_dwf_m(h, precision, psi, c, 0));
    CK(launch_reduce(precision, c, nullptr, 2L * h->g.N4h, h->Ls, h->partials, h->scal, FIN_STORE, S_TMP0, h->stream),
       "force action");
  }
  RET(ensure_gauge(h, precision));
  if (F || G)
    CK(launch_force(precision, h->c12, h->g, psi, c, h->gauge[precision][0], h->gauge[precision][1], F, G, 1.0, h->fp64_arith == GRID_DWF_FP64_ARITH_FLOAT_FLOAT,
                    h->stream),
       "force");
  RET(read_scalars(h));
  if (S_out) *S_out = h->host_scal[S_TMP0];
  return finish(h, "force");
}

int grid_dwf_pf_force(grid_dwf_t* h, const void* phi, void* X, double tol, int maxiter, int mode, int precision,
                      double* F, double* G, double* S_out, grid_dwf_cg_stats* stats) {
  const NvtxRange nvtx_("grid_dwf_pf_force");
  if (!h) return GRID_DWF_ERR_INVALID_ARG;
  if (mode < GRID_DWF_CG_FP64 || mode > GRID_DWF_CG_MIXED_BF16 || !(tol > 0) || maxiter < 0)
    return fail(h, GRID_DWF_ERR_INVALID_ARG, "pf_force: bad mode/tol/maxiter");
  if (precision != GRID_DWF_FP64 && precision != GRID_DWF_FP32)
    return fail(h, GRID_DWF_ERR_INVALID_ARG, "pf_force: precision must be FP64 or FP32");
  RET(check_ptr(h, phi, "phi"));
  RET(check_ptr(h, X, "X"));
  const size_t hb = half_bytes(h, GRID_DWF_FP64);
  if (overlap(phi, hb, X, hb)) return fail(h, GRID_DWF_ERR_ALIAS, "pf_force: X overlaps phi");
  const size_t gb = (size_t)h->g.N4h * 2 * 4 * 18 * sizeof(double);
  if (F && (overlap(F, gb, phi, hb) || overlap(F, gb, X, hb))) return fail(h, GRID_DWF_ERR_ALIAS, "pf_force: F overlaps");
  if (G && (overlap(G, gb, phi, hb) || overlap(G, gb, X, hb))) return fail(h, GRID_DWF_ERR_ALIAS, "pf_force: G overlaps");
  if (F && G && overlap(F, gb, G, gb)) return fail(h, GRID_DWF_ERR_ALIAS, "pf_force: F overlaps G");
  const auto t0 = std::chrono::steady_clock::now();
  CK(cudaStreamSynchronize(h->stream), "pf_force start");
  const long N = h->g.N4h;
  const int Ls = h->Ls;
  const int P = GRID_DWF_FP64;
  // X = (Mpc^+ Mpc)^-1 phi
  CgResult res;
  RET(cg_normal(h, phi, X, tol, maxiter, mode, res));
  // Full fields A = (Mooee^-1 D_eo X, X) and B = (Mooee^-+ (D_oe)^+ Y, Y) with Y = Mpc X:
  // dS = (1/2) Re B^+ dDhop A, i.e. -1/2 times the force kernel's bilinear.
  void *A, *B;
  RET(ws_get(h, WS_PF_A, 2 * hb, &A));
  RET(ws_get(h, WS_PF_B, 2 * hb, &B));
  char* Ae = static_cast<char*>(A);
  char* Be = static_cast<char*>(B);
  RET(mpc_impl(h, P, X, Be + hb, false, Ae));  // Ae = Mooee^-1 D_eo X, Bo = Mpc X
  RET(dhop_half(h, P, Be + hb, Be, 0, true, PRE_NONE, POST_INV_DAG, 1.0, 0.0, nullptr));
  CK(cudaMemcpyAsync(Ae + hb, X, hb, cudaMemcpyDeviceToDevice, h->stream), "pf_force copy");
  // S = Re phi^+ X (phi^+ X is real for the Hermitian positive Mpc^+ Mpc)
  CK(launch_reduce(P, phi, X, N, Ls, h->partials, h->scal, FIN_STORE, S_TMP0, h->stream), "pf_force action");
  if (F || G) {
    const void* a = A;
    const void* b = B;
    if (precision == GRID_DWF_FP32) {
      const size_t fb32 = 2 * half_bytes(h, GRID_DWF_FP32);
      void *a32, *b32;
      RET(ws_get(h, WS_PF_A32, fb32, &a32));
      RET(ws_get(h, WS_PF_B32, fb32, &b32));
      CK(launch_convert(P, GRID_DWF_FP32, A, a32, 2 * N, Ls, nullptr, 1.0, h->stream), "pf_force convert");
      CK(launch_convert(P, GRID_DWF_FP32, B, b32, 2 * N, Ls, nullptr, 1.0, h->stream), "pf_force convert");
      a = a32;
      b = b32;
    }
    RET(ensure_gauge(h, precision));
    CK(launch_force(precision, h->c12, h->g, a, b, h->gauge[precision][0], h->gauge[precision][1], F, G, -0.5, h->fp64_arith == GRID_DWF_FP64_ARITH_FLOAT_FLOAT,
                    h->stream),
       "pf_force force");
  }
  RET(read_scalars(h));
  if (S_out) *S_out = h->host_scal[S_TMP0];
  const auto t1 = std::chrono::steady_clock::now();
  if (stats) {
    stats->iterations = res.iters;
    stats->reliable_updates = res.updates;
    stats->converged = res.converged ? 1 : 0;
    stats->true_residual = res.true_res;
    stats->seconds = std::chrono::duration<double>(t1 - t0).count();
    stats->flops = res.flops + 3 * 1320.0 * (double)N * Ls;
  }
  if (!res.converged) return fail(h, GRID_DWF_ERR_NOT_CONVERGED, "pf_force: tolerance not reached within maxiter");
  return finish(h, "pf_force");
}

}  // extern "C"
