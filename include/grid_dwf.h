/*
 * grid_dwf.h -- C ABI of the GB300-native 5D domain-wall fermion operator library
 * (libgrid_dwf.so, CUDA for sm_103a).
 *
 * What it computes. The paper (Boyle et al., "Grid: OneCode and FourAPIs", LATTICE2021) names
 * the domain wall fermion (DWF) Dirac operator as the code it profiles and calls provably
 * optimal on A100 (Introduction; Section 3, the Nsight-Systems and Nsight-Compute figures; the
 * Conclusion's node-local "Wilson" matrix). It prints no formula, so the operator here is the
 * standard Shamir one:
 *   Dhop psi(x,s) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu,s) + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu,s),
 *   (Mooee psi)_s = (5 - M5) psi_s - P- psi_{s+1} - P+ psi_{s-1}, wrap terms +m P- psi_0 (s = Ls-1)
 *                   and +m P+ psi_{Ls-1} (s = 0), P+- = (1 +- gamma5)/2,
 *   M = Mooee - Dhop/2,
 * gamma matrices in the chiral basis (mu = 0..3 <-> x, y, z, t; gamma5 = diag(1, 1, -1, -1)),
 * boundary phase bc[mu] on hops that cross the lattice edge, checkerboard parity
 * (x+y+z+t) mod 2, "EO" = output even / input odd, and the odd-site Schur complement
 *   Mpc = Mooee - Moe Mooee^-1 Meo,  Meo = -D_eo/2, Moe = -D_oe/2.
 *
 * Conventions of the ABI.
 *  - Every call returns int: GRID_DWF_OK (0) or a negative GRID_DWF_ERR_* code; the message of
 *    the last failure on a handle is grid_dwf_last_error(h). No C++ exception crosses the ABI.
 *  - Field and gauge pointers are DEVICE pointers owned by the caller, 16-byte aligned, unless a
 *    call says otherwise. Calls are asynchronous on the handle's CUDA stream, except those that
 *    return a host scalar (norm2, inner, cg, force), which synchronise that stream.
 *  - Canonical layouts (FP64, complex as interleaved re, im):
 *      spinor  [t][z][y][x][s][spin 4][colour 3]        (x fastest among the 4D coordinates),
 *      gauge   [t][z][y][x][mu 4][a 3][b 3]              (row a, column b of U_mu(x)).
 *  - Device field layout (what dhop/mooee/mpc/... read and write): a half field of one parity
 *    holds V/2 checkerboard sites (cb index = lexicographic 4D index / 2). The fifth dimension
 *    is padded to Lsp = Ls rounded up to even (the pad slice is zero) and stored in slice pairs:
 *    a site holds Lsp * 24 reals as 16-byte vectors (k, q), chunk k and pair q, vector (k, q)
 *    holding reals RV*k .. RV*k+RV-1 of slices 2q and 2q+1, real-major (RV = 1, 2, 4 for FP64,
 *    FP32, FP16/BF16). Sites are grouped in blocks of 4 consecutive cb sites, and within a block
 *    the vectors are ordered [chunk k][site in block][pair q]: vector (k, q) of site i is at byte
 *    (i / 4) * 4 * S + k * 64 * Lsh + (i % 4) * 16 * Lsh + 16 * q, with Lsh = Lsp / 2 and
 *    S = 48 * Lsh * (bytes per real) the bytes of one site. A full field is the even half
 *    followed by the odd half. grid_dwf_field_bytes gives the sizes; grid_dwf_pack/unpack
 *    convert from/to canonical.
 *  - Precisions: GRID_DWF_FP64 (double storage and arithmetic), GRID_DWF_FP32 (float),
 *    GRID_DWF_FP16 and GRID_DWF_BF16 (half / bfloat16 storage, float arithmetic).
 *  - Aliasing: output buffers may not overlap inputs (GRID_DWF_ERR_ALIAS), except where a call
 *    allows in-place use.
 */
#ifndef GRID_DWF_H
#define GRID_DWF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct grid_dwf grid_dwf_t;

enum {
  GRID_DWF_OK = 0,
  GRID_DWF_ERR_INVALID_ARG = -1,
  GRID_DWF_ERR_CUDA = -2,
  GRID_DWF_ERR_OOM = -3,
  GRID_DWF_ERR_NOT_CONVERGED = -4,
  GRID_DWF_ERR_NONFINITE = -5,
  GRID_DWF_ERR_ALIAS = -6,
  GRID_DWF_ERR_NO_GAUGE = -7
};

enum { GRID_DWF_FP64 = 0, GRID_DWF_FP32 = 1, GRID_DWF_FP16 = 2, GRID_DWF_BF16 = 3 };

/* Field subsets: a half field of even or odd sites, or a full field. */
enum { GRID_DWF_EVEN = 0, GRID_DWF_ODD = 1, GRID_DWF_FULL = 2 };

/* CG modes: plain FP64, or FP64 defect correction around an inner solve whose Dirac operator and
 * search vectors are stored in FP32, FP16 or BF16 (float arithmetic), with reliable updates. */
enum { GRID_DWF_CG_FP64 = 0, GRID_DWF_CG_MIXED_FP32 = 1, GRID_DWF_CG_MIXED_FP16 = 2, GRID_DWF_CG_MIXED_BF16 = 3 };

typedef struct {
  int iterations;          /* inner (or plain) CG iterations */
  int reliable_updates;    /* FP64 true-residual recomputations (mixed modes) */
  int converged;           /* 1 if true_residual <= tol */
  double true_residual;    /* |Mpc^+ b' - Mpc^+ Mpc x_o| / |Mpc^+ b'|, recomputed in FP64 */
  double seconds;          /* wall time of the solve, measured on the host around the stream */
  double flops;            /* Dhop flops performed (1320 per 5D output site per half Dhop) */
} grid_dwf_cg_stats;

/* Create an operator on an Lx x Ly x Lz x Lt x Ls lattice.
 * dims[4] = {Lx, Ly, Lz, Lt}, each even and >= 2, Lx*Ly*Lz*Lt/2 < 2^31 / 8; 1 <= Ls <= 128;
 * M5, mass finite, and Mooee invertible for them; bc[4] each +1 (periodic) or -1
 * (antiperiodic), NULL meaning {+1, +1, +1, -1}; compress12 != 0 stores links as two rows (the
 * third rebuilt as the conjugated cross product, exact for SU(3) links); stream is a
 * cudaStream_t (NULL = legacy default stream). Uses the current CUDA device. On success *out
 * owns device memory for the links and workspaces, freed by grid_dwf_destroy.
 * Tuning read from the environment at create (the operators' results are the same bit for bit
 * and only the speed changes, except that sums over the lattice formed inside a hop, the fused
 * CG's p^+ A p and |r|^2 and the force's action, group their per-CTA partial sums differently):
 * GRID_DWF_ZBLOCK (CTA walk of the FP32/FP16/BF16 hops in blocks of that many z-planes; default:
 * 8 for FP32 when two t-planes of input, output and links exceed half of L2, else the
 * lexicographic walk, 0), GRID_DWF_PDL
 * (0 disables launching those hops as programmatic dependents of the previous kernel; default 1),
 * GRID_DWF_SITES_PER_CTA (fewer sites per CTA than fill 128 threads), GRID_DWF_SYNC_DEBUG (1:
 * synchronise after every call to surface asynchronous errors at their call). GRID_DWF_CG_LAG (0 or
 * 1) chooses whether the mixed CG decides its reliable updates on the current or the previous
 * inner residual (default 1, and 0 for BF16), which changes the iterates, not the convergence
 * criterion. GRID_DWF_CG_DELTA (a number in (0, 1)) sets the mixed CG's reliable-update threshold,
 * the factor by which the inner residual must fall before x is folded into the FP64 solution and
 * the FP64 residual recomputed (default 1e-4 for FP32 inner solves, 0.03 for FP16 and BF16). */
int grid_dwf_create(const int dims[4], int Ls, double M5, double mass, const int bc[4], int compress12, void* stream,
                    grid_dwf_t** out);
int grid_dwf_destroy(grid_dwf_t* h);
int grid_dwf_set_stream(grid_dwf_t* h, void* stream);

/* Arithmetic of the GRID_DWF_FP64 hopping term (Dhop and everything built on it: M, Mpc,
 * Mpc^+ Mpc, the FP64 CG and the FP64 true residuals of the mixed CG) and of the FP64 fermion
 * force (grid_dwf_force, grid_dwf_pf_force with precision GRID_DWF_FP64); storage stays FP64, and
 * so do the vector updates and reductions of the solvers.
 * GRID_DWF_FP64_ARITH_NATIVE (the default): IEEE double. GRID_DWF_FP64_ARITH_FLOAT_FLOAT: each
 * real carried as an unevaluated sum of two floats (Dekker's double-length arithmetic: error-free
 * TwoSum and FMA-based TwoProduct), about 46 significant bits (relative error of an operator
 * application ~1e-14) on the FP32 pipe, which on this GPU has ~64 times the FP64 pipe's
 * throughput. Its exponent range is float's: input magnitudes below 2^-103 read as zero and
 * above 2^128 as infinity. Any other mode is GRID_DWF_ERR_INVALID_ARG. Applies to calls issued
 * after it on this handle. */
enum { GRID_DWF_FP64_ARITH_NATIVE = 0, GRID_DWF_FP64_ARITH_FLOAT_FLOAT = 1 };
int grid_dwf_set_fp64_arith(grid_dwf_t* h, int mode);
const char* grid_dwf_last_error(const grid_dwf_t* h);
const char* grid_dwf_status_string(int code);

/* Bytes of a device field of the given precision and subset (half: V/2 * Lsp * 24 reals). */
int grid_dwf_field_bytes(const grid_dwf_t* h, int precision, int subset, size_t* bytes);

/* Upload the links. U is the canonical FP64 gauge field (host or device pointer; the library
 * detects which). The links are stored by the handle in every precision used later (converted
 * on first use); the boundary phase is never folded into them. */
int grid_dwf_set_gauge(grid_dwf_t* h, const double* U);

/* Canonical FP64 spinor (device, full lattice) <-> device field of `precision` for `subset`.
 * pack reads only the canonical sites of the subset; unpack writes only those sites. */
int grid_dwf_pack(grid_dwf_t* h, int precision, int subset, const double* canonical, void* field);
int grid_dwf_unpack(grid_dwf_t* h, int precision, int subset, const void* field, double* canonical);

/* Precision conversion of a device field: dst = scale * src (both of `subset`). */
int grid_dwf_convert(grid_dwf_t* h, int src_precision, int dst_precision, int subset, const void* src, void* dst,
                     double scale);

/* Hopping term. parity GRID_DWF_EVEN: out (even half) = DhopEO in (odd half); GRID_DWF_ODD:
 * out (odd) = DhopOE in (even); GRID_DWF_FULL: full fields, both halves. dag != 0: Dhop^+.
 * 1320 flops per output 5D site.
 * Source: the main DWF kernel profiled in the paper's Section 3 (Nsight-Compute figure: about 80%
 * of peak memory bandwidth, 39% of the floating-point pipe) and the Conclusion's node-local
 * "Wilson" matrix; the paper prints no formula, so the definition is the Dhop formula above
 * (chiral gamma basis, (1 - gamma_mu) on the forward hop, bc[mu] on hops crossing the edge). */
int grid_dwf_dhop(grid_dwf_t* h, int precision, const void* in, void* out, int parity, int dag);

/* Fifth-dimension operator on a field of `subset`: Mooee, Mooee^+ (dag), Mooee^-1 (inverse) or
 * (Mooee^+)^-1. In-place use (in == out) is allowed.
 * Source: one of the kernels of the DWF Dirac operator sequence in the paper's Conclusion and
 * Section 3 (Nsight-Systems figure); no formula is printed, so this is the Shamir term of the
 * preamble: (5 - M5) on the diagonal, P- coupling s to s+1 and P+ coupling s to s-1 with +m on
 * the wrap-around; Mooee^+ is its transpose in s, Mooee^-1 the closed-form inverse of the cyclic
 * bidiagonal matrix of each chirality. */
int grid_dwf_mooee(grid_dwf_t* h, int precision, int subset, const void* in, void* out, int dag, int inverse);

/* Full operator on full fields: out = M in, or M^+ in (dag).
 * Source: the DWF Dirac operator of the paper's Introduction and Section 3; the reading is
 * M = Mooee - Dhop/2 (Shamir, preamble), in one launch (Dhop with Mooee fused in). */
int grid_dwf_m(grid_dwf_t* h, int precision, const void* in, void* out, int dag);

/* Odd-site Schur complement on odd half fields: out = Mpc in (dag: Mpc^+ in). tmp_even: an even
 * half field of scratch, or NULL for a handle-owned one.
 * Source: the red-black preconditioned form in which the paper's Section 3 runs the DWF operator
 * (the Nsight-Systems "sequence" of kernels); reading: Mpc = Mooee - Moe Mooee^-1 Meo with
 * Meo = -D_eo/2, Moe = -D_oe/2, Mpc^+ = Mooee^+ - Meo^+ (Mooee^-1)^+ Moe^+ (two launches each). */
int grid_dwf_mpc(grid_dwf_t* h, int precision, const void* in, void* out, int dag, void* tmp_even);

/* out = Mpc^+ Mpc in on odd half fields. tmp_odd / tmp_even: scratch half fields or NULL.
 * Source: as grid_dwf_mpc; the Hermitian positive-definite normal operator that CG inverts
 * (four launches: each Dhop with its Mooee / Mooee^-1 step fused). */
int grid_dwf_mdagm(grid_dwf_t* h, int precision, const void* in, void* out, void* tmp_odd, void* tmp_even);

/* Reductions with FP64 accumulation, bitwise reproducible: |a|^2, and a^+ b as (re, im).
 * Source: the reduction primitive of the paper's Section 2.1 (accelerator_sum); here a fixed
 * two-pass order (608 partial sums, then one CTA) so that repeated calls agree bit for bit. */
int grid_dwf_norm2(grid_dwf_t* h, int precision, int subset, const void* a, double* result);
int grid_dwf_inner(grid_dwf_t* h, int precision, int subset, const void* a, const void* b, double result[2]);

/* Source: the paper describes no solver; this is the standard use of the operator it profiles
 * (conjugate gradient on the Schur normal equations), with these readings: stop on the FP64
 * true relative residual of the normal equations (1e-10 in the benchmarks); the mixed modes are
 * FP64 defect correction with reliable updates: the inner CG runs on vectors rescaled to unit
 * rms element, in FP32 (r, x) and the storage precision (p, A p), and the FP64 residual is
 * recomputed when the inner one has fallen by 1e-3 (FP32) or 0.03 (FP16 / BF16) since the last
 * recomputation, or when it predicts convergence.
 * Solve M x = b (full FP64 fields in device layout) through the odd-site Schur complement:
 *   b'_o = b_o - Moe Mooee^-1 b_e; CG on Mpc^+ Mpc x_o = Mpc^+ b'_o; x_e = Mooee^-1 (b_e - Meo x_o).
 * x holds the initial guess on input (its odd half is used). Stops when the FP64 true residual
 * of the normal equations falls to tol; returns GRID_DWF_ERR_NOT_CONVERGED (x and *stats still
 * filled) after maxiter iterations. stats may be NULL. */
int grid_dwf_cg(grid_dwf_t* h, const void* b, void* x, double tol, int maxiter, int mode, grid_dwf_cg_stats* stats);

/* Source: the paper describes no derivative; this is the adjoint of the operator it profiles.
 * Reading: with chi = M psi, the link derivative of S = |M psi|^2 comes from the hopping term
 * alone, per link an outer product of psi and the spin-projected chi summed over s and spin;
 * F = TA(G U^+) under U -> exp(eps A) U, TA the traceless anti-Hermitian part; FP32 fields
 * accumulate in FP32 within blocks of 16 slices and in FP64 across blocks; with FP32 fields and
 * 18-real links |M psi|^2 is summed in the launch that forms M psi (FP32 within a thread's slice
 * pair, FP64 across CTAs).
 * S = |M psi|^2 for a full field psi (FP64 or FP32), its su(3) force F and ambient gradient
 * G = dS/dRe U + i dS/dIm U, both canonical gauge layout FP64 device buffers (either may be
 * NULL). chi: full field of the same precision receiving M psi, or NULL for handle-owned
 * scratch. Under U -> exp(eps A) U with A in su(3): dS/deps = sum Re tr(A^+ F). *S_out on host. */
int grid_dwf_force(grid_dwf_t* h, int precision, const void* psi, void* chi, double* F, double* G, double* S_out);

/* Two-flavour pseudofermion action S = phi^+ (Mpc^+ Mpc)^-1 phi and its link derivative: the
 * Schur normal operator above as it enters hybrid Monte Carlo, differentiated through the solve.
 * The paper names no action; this is the next step after the operator, its solver and the force
 * of |M psi|^2 (grid_dwf_force), and reuses all three.
 *   phi        FP64 odd half field (device layout), the pseudofermion; read only.
 *   X          FP64 odd half field: initial guess on input, X = (Mpc^+ Mpc)^-1 phi on output.
 *   tol, maxiter, mode   as for grid_dwf_cg, applied to the FP64 true residual of
 *              Mpc^+ Mpc X = phi (mixed modes: inner solve in FP32/FP16/BF16 storage).
 *   precision  GRID_DWF_FP64 or GRID_DWF_FP32: arithmetic of the force contraction (FP32 fields
 *              with FP64 accumulation, as in grid_dwf_force); the solve always returns FP64 X.
 *   F, G       canonical gauge-layout FP64 device buffers (either may be NULL): the su(3) force
 *              F (dS/deps = sum Re tr(A^+ F) under U -> exp(eps A) U) and G = dS/dRe U + i dS/dIm U.
 *   S_out      host double receiving S = Re phi^+ X; stats as for grid_dwf_cg (may be NULL).
 * With Y = Mpc X, dS = -2 Re Y^+ dMpc X = (1/2) Re B^+ dDhop A for the full fields
 * A = (Mooee^-1 D_eo X, X) and B = (Mooee^-+ (D_oe)^+ Y, Y), contracted by the force kernel.
 * Synchronises the handle's stream. Returns GRID_DWF_ERR_NOT_CONVERGED (X, F, G, S and stats
 * still written) if tol is not reached within maxiter. */
int grid_dwf_pf_force(grid_dwf_t* h, const void* phi, void* X, double tol, int maxiter, int mode, int precision,
                      double* F, double* G, double* S_out, grid_dwf_cg_stats* stats);

/* A lattice split into blocks along t (one block per handle: dims[3] is the block's extent, even,
 * its first t-plane at an even global t). Source: the paper's Section 3, whose multi-GPU runs
 * assemble the faces of each GPU's block in their own kernels and overlap the exchange with the
 * interior of the hopping term. Per hop of output parity p, each block
 *   - projects its input half field (parity 1 - p) on its first t-plane with the forward-hop
 *     projector and on its last t-plane with the backward-hop projector (grid_dwf_face_project;
 *     phase_first / phase_last: the boundary phase bc[t] if that face crosses the global lattice
 *     edge, else +1; dag as for the hop), and sends send_first to the previous block and
 *     send_last to the next one (the caller moves them, e.g. by peer copies into local buffers);
 *   - computes its interior (all output sites off the two face planes: their neighbours are local)
 *     with grid_dwf_dhop_region(..., GRID_DWF_REGION_INTERIOR, NULL, NULL, NULL) while the faces
 *     travel, then its two face planes with GRID_DWF_REGION_FACES, recv_fwd = the next block's
 *     send_first, recv_bwd = the previous block's send_last, links_bwd = the previous block's
 *     grid_dwf_face_links(prec, p) (the links U_t of its last plane, exchanged once per gauge field).
 * Faces are FP32 half spinors, [face site][6][slice pair] 16-byte vectors, face site = cb index
 * within the t-plane (grid_dwf_face_bytes gives the size, link faces are in the stored link
 * format); the result equals the hop of the whole lattice bit for bit. FP32, FP16 and BF16 fields;
 * each t-plane must hold whole CTAs of sites (GRID_DWF_ERR_INVALID_ARG otherwise). */
enum { GRID_DWF_REGION_INTERIOR = 0, GRID_DWF_REGION_FACES = 1 };
int grid_dwf_face_bytes(const grid_dwf_t* h, int precision, size_t* face_bytes, size_t* link_face_bytes);
int grid_dwf_face_project(grid_dwf_t* h, int precision, const void* in, int dag, int phase_first, int phase_last,
                          void* send_first, void* send_last);
int grid_dwf_face_links(grid_dwf_t* h, int precision, int out_parity, void* links_last);
int grid_dwf_dhop_region(grid_dwf_t* h, int precision, const void* in, void* out, int out_parity, int dag,
                         int region, const void* recv_fwd, const void* recv_bwd, const void* links_bwd);

/* Measured arithmetic ceiling of the current device, the denominator of the roofline of a kernel
 * bound by its arithmetic pipe rather than by memory (the IEEE FP64 hopping term on this GPU):
 * FP64 FMA, scalar FP32 FMA or packed FP32x2 FMA throughput, in GFLOP/s (2 flops per FMA, 4 per
 * packed FMA) over all SMs, the best of three timed throughput loops (independent FMA chains,
 * 8 CTAs of 256 threads per SM) after one warm-up, on `stream` (NULL = legacy default stream).
 * Not part of the paper's method: a measurement service (the paper's Section 3 reports its
 * kernel's floating-point pipe utilisation, 39%, against such a ceiling). Synchronises the
 * stream; allocates nothing. */
enum { GRID_DWF_PEAK_FP64_FMA = 0, GRID_DWF_PEAK_FP32_FMA = 1, GRID_DWF_PEAK_FP32X2_FMA = 2 };
int grid_dwf_pipe_peak(int kind, void* stream, double* gflops);

/* Software-managed device cache of host fields, for workloads whose fields do not all fit in the
 * GPU's memory. Source: the paper's Section 2.3 ("Memory models and software managed cache"):
 * host data moved to the device when a view is opened with an access intent, a device footprint
 * capped by a high watermark, least-recently-used replacement under the program's control, and an
 * "advise" priority for large, rarely used fields. The cache is independent of the operator
 * handle: a caller opens views on its host fields and passes the returned device pointers to the
 * operator calls (which must complete, on the cache's stream or after it, before the view's data
 * is evicted: close views only when the kernels that use them are queued behind later cache
 * traffic on the same stream, or synchronise).
 *   create   high_watermark: the most device bytes the cache may hold; stream: cudaStream_t of its
 *            copies (NULL = legacy default stream); backend: NULL for CUDA (cudaMalloc, cudaFree,
 *            cudaMemcpyAsync; host buffers should be pinned), or caller functions (each returns 0
 *            on success) that move data, e.g. to exercise the cache without a GPU.
 *   open     the field is the host buffer `host` of `bytes` bytes (registered on first open; the
 *            same size on every open). Intents: GRID_DWF_ACC_READ (device copy made current),
 *            GRID_DWF_ACC_WRITE (made current, then marked newer than the host's),
 *            GRID_DWF_ACC_WRITE_DISCARD (device buffer provided, not filled, marked newer),
 *            GRID_DWF_CPU_READ (host copy made current; *ptr = host), GRID_DWF_CPU_WRITE (host copy
 *            made current and marked newer). An accelerator open returns the device pointer and
 *            pins it until the matching close; if the new device buffer does not fit under the
 *            watermark, unpinned fields are evicted from the back of the LRU order (fields advised
 *            GRID_DWF_ADVISE_INFREQUENT first), a newer device copy written back before it is freed;
 *            GRID_DWF_ERR_OOM if pinned fields leave no room. A CPU open while accelerator views
 *            are open is GRID_DWF_ERR_ALIAS. CPU opens synchronise the cache's stream.
 *   flush    writes every newer, unpinned device copy back to the host (the copies stay).
 *   forget   writes back and drops one field's entry and device buffer.
 *   query    the entry's state (0 empty: no device copy, 1 consistent, 2 host newer, 3 device
 *            newer), its open accelerator views and device pointer (for tests and tools).
 * A cache is not safe for concurrent calls from several host threads; use one per thread or
 * serialise the calls. */
typedef struct grid_dwf_cache grid_dwf_cache_t;
enum { GRID_DWF_CPU_READ = 0, GRID_DWF_CPU_WRITE = 1, GRID_DWF_ACC_READ = 2, GRID_DWF_ACC_WRITE = 3,
       GRID_DWF_ACC_WRITE_DISCARD = 4 };
enum { GRID_DWF_ADVISE_NORMAL = 0, GRID_DWF_ADVISE_INFREQUENT = 1 };
typedef struct {
  void* ctx;
  int (*alloc)(void* ctx, size_t bytes, void** dev);
  int (*free)(void* ctx, void* dev);
  int (*to_device)(void* ctx, void* dev, const void* host, size_t bytes);
  int (*to_host)(void* ctx, void* host, const void* dev, size_t bytes);
} grid_dwf_cache_backend;
typedef struct {
  unsigned long long hits, misses, evictions, cpu_opens;
  unsigned long long copies_to_device, copies_to_host, bytes_to_device, bytes_to_host;
  size_t peak_resident, resident_bytes;
} grid_dwf_cache_stats;
int grid_dwf_cache_create(size_t high_watermark, void* stream, const grid_dwf_cache_backend* backend,
                          grid_dwf_cache_t** out);
int grid_dwf_cache_destroy(grid_dwf_cache_t* c);
int grid_dwf_cache_advise(grid_dwf_cache_t* c, void* host, size_t bytes, int advice);
int grid_dwf_cache_open(grid_dwf_cache_t* c, void* host, size_t bytes, int intent, void** ptr);
int grid_dwf_cache_close(grid_dwf_cache_t* c, void* host);
int grid_dwf_cache_flush(grid_dwf_cache_t* c);
int grid_dwf_cache_forget(grid_dwf_cache_t* c, void* host);
int grid_dwf_cache_query(const grid_dwf_cache_t* c, const void* host, int* state, int* views, void** dev);
int grid_dwf_cache_get_stats(const grid_dwf_cache_t* c, grid_dwf_cache_stats* st);
const char* grid_dwf_cache_last_error(const grid_dwf_cache_t* c);

/* |a|^2 (b == NULL) or a^+ b with FP64 accumulation, like grid_dwf_norm2 / grid_dwf_inner, for
 * callers that cannot allocate device memory: code recording a CUDA graph (where cudaMalloc is
 * not allowed), loops that must not take cudaMalloc's implicit device synchronisation, or a host
 * framework that owns all device memory through its own pool and has none to spare. It needs no
 * handle and allocates nothing: its scratch (partial sums) is a fixed 256 KiB array in the
 * library's device image, present on every GPU that loads the library until the process exits.
 * The paper has no counterpart; this is a service of the library.
 *   a, b      device fields of `precision` in the device layout (16-byte aligned), nsites
 *             checkerboard sites of Ls slices each, padded to even as in every field of this
 *             library (V/2 sites for a half field, V for a full one). nsites must be a multiple
 *             of 4, since the layout stores sites in blocks of 4 (every half field of an even
 *             lattice is); any other nsites is GRID_DWF_ERR_INVALID_ARG before any launch;
 *   result    device pointer to 2 doubles (8-byte aligned), receives (re, im) (im = 0 for |a|^2);
 *   stream    cudaStream_t the two kernels run on (NULL = legacy default stream); asynchronous;
 *   err       optional buffer for a message on failure.
 * Limit: nsites * Lsp <= 22369620 five-dimensional sites, Lsp = Ls rounded up to even (e.g. a
 * 32^4 x 16 full field, 16777216); larger fields are rejected with GRID_DWF_ERR_INVALID_ARG
 * before anything runs. The first call
 * on a device looks up the array's device address (once per device, with that device current);
 * make that first call before any stream capture. The address is cached per device index for the
 * life of the process: the library assumes the device's primary context (the one the CUDA
 * runtime uses) and no cudaDeviceReset between calls, since a reset or a different context
 * would leave the cached address stale. All calls share the one array, which keeps the
 * last call's partial sums (each call overwrites what it reads), so calls whose kernels overlap
 * on the GPU (on different streams, or different host threads) race and give wrong results. */
int grid_dwf_inner_noalloc(int precision, const void* a, const void* b, long nsites, int Ls, void* stream,
                           double* result, char* err, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* GRID_DWF_H */
