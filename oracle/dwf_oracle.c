/*
 * dwf_oracle.c -- plain FP64 CPU oracle for the 5D Shamir domain-wall fermion operator.
 *
 * TEST INFRASTRUCTURE. This is the slow, obviously correct reference that the CUDA library is
 * checked against. Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it. It shares no code, header, table or constant with the CUDA library, and
 * the library never calls it.
 *
 * What the paper fixes and what it leaves open. The paper (Introduction; Section 3, the
 * Nsight-Compute profile of its main DWF kernel and the Conclusion's node-local
 * "Wilson" matrix) names the domain wall fermion Dirac operator and its Wilson hopping kernel
 * as the memory-bound hot path, but prints no formula for them. The oracle therefore writes
 * out the standard Shamir operator, with these readings:
 *   - gamma matrices in the chiral basis, mu = 0,1,2,3 <-> x,y,z,t:
 *       gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = x,y,z), gamma_t = [[0, 1], [1, 0]],
 *       gamma5 = gamma_x gamma_y gamma_z gamma_t = diag(1, 1, -1, -1);
 *   - Dhop psi(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu),
 *     the same for every fifth-dimension slice s; Dhop^+ swaps the two projector signs;
 *   - boundary phase bc[mu] (+1 periodic, -1 antiperiodic) on every hop that crosses the
 *     lattice edge in direction mu; it is never folded into the stored links;
 *   - Mooee (the part of M that is local in 4D and couples s):
 *       (Mooee psi)_s = (5 - M5) psi_s - P- psi_{s+1} - P+ psi_{s-1},
 *     with P+- = (1 +- gamma5)/2 and the wrap-around terms +m P- psi_0 (at s = Ls-1) and
 *     +m P+ psi_{Ls-1} (at s = 0) in place of the missing neighbours;
 *   - M = Mooee - Dhop/2; even/odd from (x+y+z+t) mod 2; "EO" = output even, input odd;
 *     Schur complement on odd sites Mpc = Mooee - Moe Mooee^-1 Meo, Meo = -D_eo/2, Moe = -D_oe/2.
 *
 * Layouts (all FP64, complex numbers as interleaved (re, im) pairs):
 *   spinor  psi[site][s][spin 4][colour 3], site = x + Lx*(y + Ly*(z + Lz*t));
 *   gauge   U[site][mu 4][a 3][b 3], row a, column b of U_mu(site).
 * A half-lattice field is held as a full-size array; the oracle reads only the sites of the
 * parity it needs and writes zero on the other parity.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
  int L[4];
  int Ls;
  int bc[4];
  long V;
} geom_t;

static geom_t make_geom(const int dims[4], int Ls, const int bc[4]) {
  geom_t g;
  g.V = 1;
  for (int m = 0; m < 4; ++m) {
    g.L[m] = dims[m];
    g.bc[m] = bc ? bc[m] : 1;
    g.V *= dims[m];
  }
  g.Ls = Ls;
  return g;
}

static long lex_index(const geom_t* g, const int c[4]) {
  return c[0] + (long)g->L[0] * (c[1] + (long)g->L[1] * (c[2] + (long)g->L[2] * c[3]));
}

static void site_coords(const geom_t* g, long site, int c[4]) {
  for (int m = 0; m < 4; ++m) {
    c[m] = (int)(site % g->L[m]);
    site /= g->L[m];
  }
}

static int site_parity(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

/* gamma_x, gamma_y, gamma_z, gamma_t and gamma5, built from the Pauli matrices. */
static void gamma_matrices(cplx g[5][4][4]) {
  const cplx iu = _Complex_I;
  const cplx sigma[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -iu}, {iu, 0}}, {{1, 0}, {0, -1}}};
  memset(g, 0, sizeof(cplx) * 5 * 16);
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        g[k][a][2 + b] = -iu * sigma[k][a][b];
        g[k][2 + a][b] = iu * sigma[k][a][b];
      }
  for (int a = 0; a < 2; ++a) {
    g[3][a][2 + a] = 1;
    g[3][2 + a][a] = 1;
  }
  cplx t1[4][4], t2[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      t1[i][j] = 0;
      for (int k = 0; k < 4; ++k) t1[i][j] += g[0][i][k] * g[1][k][j];
    }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      t2[i][j] = 0;
      for (int k = 0; k < 4; ++k) t2[i][j] += t1[i][k] * g[2][k][j];
    }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      g[4][i][j] = 0;
      for (int k = 0; k < 4; ++k) g[4][i][j] += t2[i][k] * g[3][k][j];
    }
}

/* Exported for the tests: gamma_x..gamma_t, gamma5 as [5][4][4] complex. */
void dwf_oracle_gamma(double* out) {
  cplx g[5][4][4];
  gamma_matrices(g);
  memcpy(out, g, sizeof(g));
}

/*
 * Wilson hopping term at one 4D site x, every slice s (the "node local Wilson matrix" of the
 * paper's Conclusion, acting on a 5D field): o[s][spin][colour] = (Dhop in)(x, s), or Dhop^+.
 */
static void dhop_site(const geom_t* g, cplx gam[5][4][4], const cplx* U, const cplx* in, long x, int dag, cplx* o) {
  int c[4];
  site_coords(g, x, c);
  /* Forward hop projector (1 - gamma), backward (1 + gamma); the adjoint swaps them. */
  const double fwd_sign = dag ? +1.0 : -1.0;
  const double bwd_sign = -fwd_sign;
  for (int s = 0; s < g->Ls; ++s) {
    cplx acc[12] = {0};
    for (int mu = 0; mu < 4; ++mu) {
      for (int dir = 0; dir < 2; ++dir) {
        int cn[4] = {c[0], c[1], c[2], c[3]};
        double phase = 1.0;
        long link_site;
        if (dir == 0) { /* x + mu, link U_mu(x) */
          if (c[mu] == g->L[mu] - 1) phase = g->bc[mu];
          cn[mu] = (c[mu] + 1) % g->L[mu];
          link_site = x;
        } else { /* x - mu, link U_mu(x - mu)^+ */
          if (c[mu] == 0) phase = g->bc[mu];
          cn[mu] = (c[mu] - 1 + g->L[mu]) % g->L[mu];
          link_site = lex_index(g, cn);
        }
        const long xn = lex_index(g, cn);
        const cplx* p = in + (xn * g->Ls + s) * 12;
        const cplx* u = U + (link_site * 4 + mu) * 9;
        cplx v[12];
        for (int sp = 0; sp < 4; ++sp)
          for (int a = 0; a < 3; ++a) {
            cplx t = 0;
            for (int b = 0; b < 3; ++b) t += (dir == 0 ? u[a * 3 + b] : conj(u[b * 3 + a])) * p[sp * 3 + b];
            v[sp * 3 + a] = t;
          }
        const double gs = dir == 0 ? fwd_sign : bwd_sign;
        for (int sp = 0; sp < 4; ++sp)
          for (int a = 0; a < 3; ++a) {
            cplx gv = 0;
            for (int sq = 0; sq < 4; ++sq) gv += gam[mu][sp][sq] * v[sq * 3 + a];
            acc[sp * 3 + a] += phase * (v[sp * 3 + a] + gs * gv);
          }
      }
    }
    for (int i = 0; i < 12; ++i) o[s * 12 + i] = acc[i];
  }
}

/*
 * Wilson hopping term on the whole lattice. out_parity 0 or 1 computes only the output sites of
 * that parity (DhopEO for 0, DhopOE for 1; the inputs read are then automatically of the other
 * parity) and writes zero on the rest; 2 computes every site. dag selects Dhop^+.
 */
void dwf_oracle_dhop(const int dims[4], int Ls, const int bc[4], const double* Ud, const double* ind,
                     double* outd, int out_parity, int dag, int nthreads) {
  const geom_t g = make_geom(dims, Ls, bc);
  cplx gam[5][4][4];
  gamma_matrices(gam);
  const cplx* U = (const cplx*)Ud;
  const cplx* in = (const cplx*)ind;
  cplx* out = (cplx*)outd;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (long x = 0; x < g.V; ++x) {
    int c[4];
    site_coords(&g, x, c);
    cplx* o = out + x * g.Ls * 12;
    if (out_parity != 2 && site_parity(c) != out_parity) {
      for (int i = 0; i < g.Ls * 12; ++i) o[i] = 0;
      continue;
    }
    dhop_site(&g, gam, U, in, x, dag, o);
  }
}

/*
 * The same hopping term at a list of 4D sites only (lexicographic indices): out[k][s][spin][colour]
 * = (Dhop in)(sites[k], s). Lets large lattices be checked, and timed, on a sample of sites.
 */
void dwf_oracle_dhop_sites(const int dims[4], int Ls, const int bc[4], const double* Ud, const double* ind,
                           const long* sites, long nsites, double* outd, int dag, int nthreads) {
  const geom_t g = make_geom(dims, Ls, bc);
  cplx gam[5][4][4];
  gamma_matrices(gam);
  const cplx* U = (const cplx*)Ud;
  const cplx* in = (const cplx*)ind;
  cplx* out = (cplx*)outd;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (long k = 0; k < nsites; ++k) dhop_site(&g, gam, U, in, sites[k], dag, out + k * g.Ls * 12);
}

/* The (4 Ls) x (4 Ls) matrix of Mooee on one 4D site and one colour, index (s, spin). */
static void build_mooee_matrix(int Ls, double M5, double mass, cplx* K) {
  cplx gam[5][4][4];
  gamma_matrices(gam);
  double Pp[4][4], Pm[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      const double id = a == b ? 1.0 : 0.0;
      Pp[a][b] = 0.5 * (id + creal(gam[4][a][b]));
      Pm[a][b] = 0.5 * (id - creal(gam[4][a][b]));
    }
  const int n = 4 * Ls;
  for (int i = 0; i < n * n; ++i) K[i] = 0;
  for (int s = 0; s < Ls; ++s)
    for (int a = 0; a < 4; ++a) {
      const int row = s * 4 + a;
      K[row * n + row] += 5.0 - M5;
      for (int b = 0; b < 4; ++b) {
        if (s < Ls - 1)
          K[row * n + (s + 1) * 4 + b] -= Pm[a][b];
        else
          K[row * n + 0 * 4 + b] += mass * Pm[a][b];
        if (s > 0)
          K[row * n + (s - 1) * 4 + b] -= Pp[a][b];
        else
          K[row * n + (Ls - 1) * 4 + b] += mass * Pp[a][b];
      }
    }
}

/* Inverse by Gauss-Jordan elimination with partial pivoting. Returns 0, or -1 if singular. */
static int invert_matrix(int n, const cplx* A, cplx* Ainv) {
  cplx* W = (cplx*)malloc(sizeof(cplx) * n * 2 * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) W[i * 2 * n + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (cabs(W[r * 2 * n + col]) > cabs(W[piv * 2 * n + col])) piv = r;
    if (cabs(W[piv * 2 * n + col]) == 0.0) {
      free(W);
      return -1;
    }
    if (piv != col)
      for (int j = 0; j < 2 * n; ++j) {
        cplx t = W[col * 2 * n + j];
        W[col * 2 * n + j] = W[piv * 2 * n + j];
        W[piv * 2 * n + j] = t;
      }
    const cplx d = W[col * 2 * n + col];
    for (int j = 0; j < 2 * n; ++j) W[col * 2 * n + j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const cplx f = W[r * 2 * n + col];
      if (f == 0) continue;
      for (int j = 0; j < 2 * n; ++j) W[r * 2 * n + j] -= f * W[col * 2 * n + j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = W[i * 2 * n + n + j];
  free(W);
  return 0;
}

/*
 * Mooee and its relatives on every 4D site: inverse 0 applies Mooee (dag: Mooee^+), inverse 1
 * applies Mooee^-1 (dag: (Mooee^+)^-1), the inverse taken by Gauss-Jordan elimination of the
 * 4Ls x 4Ls matrix above. Returns -1 if that matrix is singular.
 */
int dwf_oracle_mooee(const int dims[4], int Ls, double M5, double mass, const double* ind, double* outd,
                     int dag, int inverse, int nthreads) {
  const geom_t g = make_geom(dims, Ls, NULL);
  const int n = 4 * Ls;
  cplx* K = (cplx*)malloc(sizeof(cplx) * n * n);
  cplx* Op = (cplx*)malloc(sizeof(cplx) * n * n);
  build_mooee_matrix(Ls, M5, mass, K);
  int rc = 0;
  if (inverse) {
    cplx* Ki = (cplx*)malloc(sizeof(cplx) * n * n);
    rc = invert_matrix(n, K, Ki);
    memcpy(K, Ki, sizeof(cplx) * n * n);
    free(Ki);
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Op[i * n + j] = dag ? conj(K[j * n + i]) : K[i * n + j];
  const cplx* in = (const cplx*)ind;
  cplx* out = (cplx*)outd;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (long x = 0; x < g.V; ++x) {
    const cplx* p = in + x * Ls * 12;
    cplx* o = out + x * Ls * 12;
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < n; ++i) {
        cplx t = 0;
        for (int j = 0; j < n; ++j) t += Op[i * n + j] * p[j * 3 + a];
        o[i * 3 + a] = t;
      }
  }
  free(K);
  free(Op);
  return rc;
}

static void zero_parity(const geom_t* g, cplx* f, int parity) {
  for (long x = 0; x < g->V; ++x) {
    int c[4];
    site_coords(g, x, c);
    if (site_parity(c) == parity)
      for (int i = 0; i < g->Ls * 12; ++i) f[x * g->Ls * 12 + i] = 0;
  }
}

/* The full (unpreconditioned) operator M = Mooee - Dhop/2; dag gives M^+ = Mooee^+ - Dhop^+/2. */
void dwf_oracle_m(const int dims[4], int Ls, double M5, double mass, const int bc[4], const double* U,
                  const double* in, double* out, int dag, int nthreads) {
  const geom_t g = make_geom(dims, Ls, bc);
  const long n = g.V * Ls * 12;
  cplx* t = (cplx*)malloc(sizeof(cplx) * n);
  dwf_oracle_dhop(dims, Ls, bc, U, in, (double*)t, 2, dag, nthreads);
  dwf_oracle_mooee(dims, Ls, M5, mass, in, out, dag, 0, nthreads);
  cplx* o = (cplx*)out;
  for (long i = 0; i < n; ++i) o[i] -= 0.5 * t[i];
  free(t);
}

/*
 * Schur complement on the odd sites, Mpc = Mooee - Moe Mooee^-1 Meo = Mooee - D_oe Mooee^-1 D_eo / 4,
 * and (dag) Mpc^+ = Mooee^+ - (D^+)_oe (Mooee^+)^-1 (D^+)_eo / 4. Reads the odd sites of in and
 * writes the odd sites of out (even sites of out set to zero).
 */
void dwf_oracle_mpc(const int dims[4], int Ls, double M5, double mass, const int bc[4], const double* U,
                    const double* in, double* out, int dag, int nthreads) {
  const geom_t g = make_geom(dims, Ls, bc);
  const long n = g.V * Ls * 12;
  cplx* t1 = (cplx*)malloc(sizeof(cplx) * n);
  cplx* t2 = (cplx*)malloc(sizeof(cplx) * n);
  cplx* in_odd = (cplx*)malloc(sizeof(cplx) * n);
  memcpy(in_odd, in, sizeof(cplx) * n);
  zero_parity(&g, in_odd, 0);
  dwf_oracle_dhop(dims, Ls, bc, U, (const double*)in_odd, (double*)t1, 0, dag, nthreads);
  dwf_oracle_mooee(dims, Ls, M5, mass, (const double*)t1, (double*)t2, dag, 1, nthreads);
  dwf_oracle_dhop(dims, Ls, bc, U, (const double*)t2, (double*)t1, 1, dag, nthreads);
  dwf_oracle_mooee(dims, Ls, M5, mass, (const double*)in_odd, out, dag, 0, nthreads);
  cplx* o = (cplx*)out;
  for (long i = 0; i < n; ++i) o[i] -= 0.25 * t1[i];
  zero_parity(&g, o, 0);
  free(t1);
  free(t2);
  free(in_odd);
}

/* Mpc^+ Mpc on the odd sites. */
void dwf_oracle_mdagm(const int dims[4], int Ls, double M5, double mass, const int bc[4], const double* U,
                      const double* in, double* out, int nthreads) {
  const geom_t g = make_geom(dims, Ls, bc);
  const long n = g.V * Ls * 12;
  cplx* t = (cplx*)malloc(sizeof(cplx) * n);
  dwf_oracle_mpc(dims, Ls, M5, mass, bc, U, in, (double*)t, 0, nthreads);
  dwf_oracle_mpc(dims, Ls, M5, mass, bc, U, (const double*)t, out, 1, nthreads);
  free(t);
}

static double norm2(long n, const cplx* v) {
  double s = 0;
  for (long i = 0; i < n; ++i) s += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
  return s;
}

static cplx inner(long n, const cplx* a, const cplx* b) {
  cplx s = 0;
  for (long i = 0; i < n; ++i) s += conj(a[i]) * b[i];
  return s;
}

double dwf_oracle_norm2(long n_complex, const double* v) { return norm2(n_complex, (const cplx*)v); }

void dwf_oracle_inner(long n_complex, const double* a, const double* b, double* out_re_im) {
  const cplx s = inner(n_complex, (const cplx*)a, (const cplx*)b);
  out_re_im[0] = creal(s);
  out_re_im[1] = cimag(s);
}

/*
 * Solve M x = b through the Schur complement on odd sites:
 *   b'_o = b_o - Moe Mooee^-1 b_e,   CG on Mpc^+ Mpc x_o = Mpc^+ b'_o,   x_e = Mooee^-1 (b_e - Meo x_o).
 * Plain conjugate gradients (Hestenes-Stiefel) from the initial guess in x (odd sites), stopping
 * when |r| <= tol |Mpc^+ b'| on the recursively updated residual. Writes the iteration count and
 * the true relative residual of the normal equations, recomputed at the end.
 */
int dwf_oracle_schur_cg(const int dims[4], int Ls, double M5, double mass, const int bc[4], const double* U,
                        const double* bd, double* xd, double tol, int maxiter, int* iters, double* true_resid,
                        int nthreads) {
  const geom_t g = make_geom(dims, Ls, bc);
  const long n = g.V * Ls * 12;
  const cplx* b = (const cplx*)bd;
  cplx* x = (cplx*)xd;
  cplx* t1 = (cplx*)calloc(n, sizeof(cplx));
  cplx* t2 = (cplx*)calloc(n, sizeof(cplx));
  cplx* bp = (cplx*)calloc(n, sizeof(cplx));
  cplx* rhs = (cplx*)calloc(n, sizeof(cplx));
  cplx* r = (cplx*)calloc(n, sizeof(cplx));
  cplx* p = (cplx*)calloc(n, sizeof(cplx));
  cplx* Ap = (cplx*)calloc(n, sizeof(cplx));
  /* b'_o = b_o + D_oe Mooee^-1 b_e / 2 */
  memcpy(t1, b, sizeof(cplx) * n);
  zero_parity(&g, t1, 1);
  dwf_oracle_mooee(dims, Ls, M5, mass, (const double*)t1, (double*)t2, 0, 1, nthreads);
  dwf_oracle_dhop(dims, Ls, bc, U, (const double*)t2, (double*)t1, 1, 0, nthreads);
  for (long i = 0; i < n; ++i) bp[i] = b[i] + 0.5 * t1[i];
  zero_parity(&g, bp, 0);
  dwf_oracle_mpc(dims, Ls, M5, mass, bc, U, (const double*)bp, (double*)rhs, 1, nthreads);
  zero_parity(&g, x, 0);
  dwf_oracle_mdagm(dims, Ls, M5, mass, bc, U, (const double*)x, (double*)Ap, nthreads);
  for (long i = 0; i < n; ++i) {
    r[i] = rhs[i] - Ap[i];
    p[i] = r[i];
  }
  const double rhs_norm = sqrt(norm2(n, rhs));
  double rr = norm2(n, r);
  int k = 0;
  int rc = 0;
  while (sqrt(rr) > tol * rhs_norm) {
    if (k >= maxiter) {
      rc = 1;
      break;
    }
    dwf_oracle_mdagm(dims, Ls, M5, mass, bc, U, (const double*)p, (double*)Ap, nthreads);
    const double pAp = creal(inner(n, p, Ap));
    const double alpha = rr / pAp;
    for (long i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
    }
    const double rr_new = norm2(n, r);
    const double beta = rr_new / rr;
    rr = rr_new;
    for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    ++k;
  }
  dwf_oracle_mdagm(dims, Ls, M5, mass, bc, U, (const double*)x, (double*)Ap, nthreads);
  for (long i = 0; i < n; ++i) r[i] = rhs[i] - Ap[i];
  *true_resid = sqrt(norm2(n, r)) / rhs_norm;
  *iters = k;
  /* x_e = Mooee^-1 (b_e + D_eo x_o / 2) */
  dwf_oracle_dhop(dims, Ls, bc, U, (const double*)x, (double*)t1, 0, 0, nthreads);
  for (long i = 0; i < n; ++i) t1[i] = b[i] + 0.5 * t1[i];
  zero_parity(&g, t1, 1);
  dwf_oracle_mooee(dims, Ls, M5, mass, (const double*)t1, (double*)t2, 0, 1, nthreads);
  for (long xs = 0; xs < g.V; ++xs) {
    int c[4];
    site_coords(&g, xs, c);
    if (site_parity(c) == 0)
      for (int i = 0; i < Ls * 12; ++i) x[xs * Ls * 12 + i] = t2[xs * Ls * 12 + i];
  }
  free(t1);
  free(t2);
  free(bp);
  free(rhs);
  free(r);
  free(p);
  free(Ap);
  return rc;
}

/* Traceless anti-Hermitian part, TA(X) = (X - X^+)/2 - tr(X - X^+)/6. */
static void traceless_antihermitian(const cplx X[9], cplx out[9]) {
  cplx tr = 0;
  for (int a = 0; a < 3; ++a) tr += X[a * 3 + a] - conj(X[a * 3 + a]);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) out[a * 3 + b] = 0.5 * (X[a * 3 + b] - conj(X[b * 3 + a])) - (a == b ? tr / 6.0 : 0);
}

/*
 * Action S = |M psi|^2 and its derivatives with respect to the links, with chi = M psi.
 * Per link U_mu(x), with phase the boundary factor of the hop x -> x+mu:
 *   B1 = sum_{s,spin} psi(x+mu) (x) [(1 - gamma_mu) chi(x)]^+,
 *   B2 = sum_{s,spin} psi(x) (x) [(1 + gamma_mu) chi(x+mu)]^+          (colour outer products),
 *   G  = dS/dRe U + i dS/dIm U = -phase (B1^+ + B2)                    (ambient gradient),
 *   Y  = phase (-U B1 + B2 U^+),   F = -TA(Y)                          (su(3) force),
 * so that under U -> exp(eps A) U, A in su(3), dS/deps = Re tr(A^+ F). G and F may be NULL.
 * Returns S.
 */
double dwf_oracle_force(const int dims[4], int Ls, double M5, double mass, const int bc[4], const double* Ud,
                        const double* psid, double* Fd, double* Gd, int nthreads) {
  const geom_t g = make_geom(dims, Ls, bc);
  const long n = g.V * Ls * 12;
  cplx gam[5][4][4];
  gamma_matrices(gam);
  cplx* chi = (cplx*)malloc(sizeof(cplx) * n);
  dwf_oracle_m(dims, Ls, M5, mass, bc, Ud, psid, (double*)chi, 0, nthreads);
  const double S = norm2(n, chi);
  const cplx* U = (const cplx*)Ud;
  const cplx* psi = (const cplx*)psid;
  cplx* F = (cplx*)Fd;
  cplx* G = (cplx*)Gd;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (long x = 0; x < g.V; ++x) {
    int c[4];
    site_coords(&g, x, c);
    for (int mu = 0; mu < 4; ++mu) {
      int cn[4] = {c[0], c[1], c[2], c[3]};
      cn[mu] = (c[mu] + 1) % g.L[mu];
      const long xf = lex_index(&g, cn);
      const double phase = c[mu] == g.L[mu] - 1 ? g.bc[mu] : 1.0;
      cplx B1[9] = {0}, B2[9] = {0};
      for (int s = 0; s < Ls; ++s) {
        const cplx* psi_x = psi + (x * Ls + s) * 12;
        const cplx* psi_f = psi + (xf * Ls + s) * 12;
        const cplx* chi_x = chi + (x * Ls + s) * 12;
        const cplx* chi_f = chi + (xf * Ls + s) * 12;
        cplx w1[12], w2[12];
        for (int sp = 0; sp < 4; ++sp)
          for (int a = 0; a < 3; ++a) {
            cplx g1 = 0, g2 = 0;
            for (int sq = 0; sq < 4; ++sq) {
              g1 += gam[mu][sp][sq] * chi_x[sq * 3 + a];
              g2 += gam[mu][sp][sq] * chi_f[sq * 3 + a];
            }
            w1[sp * 3 + a] = chi_x[sp * 3 + a] - g1;
            w2[sp * 3 + a] = chi_f[sp * 3 + a] + g2;
          }
        for (int sp = 0; sp < 4; ++sp)
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              B1[a * 3 + b] += psi_f[sp * 3 + a] * conj(w1[sp * 3 + b]);
              B2[a * 3 + b] += psi_x[sp * 3 + a] * conj(w2[sp * 3 + b]);
            }
      }
      const cplx* u = U + (x * 4 + mu) * 9;
      cplx Y[9];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          cplx uB1 = 0, B2ud = 0;
          for (int k = 0; k < 3; ++k) {
            uB1 += u[a * 3 + k] * B1[k * 3 + b];
            B2ud += B2[a * 3 + k] * conj(u[b * 3 + k]);
          }
          Y[a * 3 + b] = phase * (-uB1 + B2ud);
        }
      if (F) {
        cplx ta[9];
        traceless_antihermitian(Y, ta);
        for (int i = 0; i < 9; ++i) F[(x * 4 + mu) * 9 + i] = -ta[i];
      }
      if (G)
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) G[(x * 4 + mu) * 9 + a * 3 + b] = -phase * (conj(B1[b * 3 + a]) + B2[a * 3 + b]);
    }
  }
  free(chi);
  return S;
}

/*
 * Two-flavour pseudofermion action on odd sites, S = phi^+ (Mpc^+ Mpc)^-1 phi, and its
 * derivative with respect to the links: the action that hybrid Monte Carlo integrates,
 * differentiated through the solve.
 *
 * X = (Mpc^+ Mpc)^-1 phi by plain conjugate gradients from X = 0, stopping when the recursive
 * residual satisfies |r| <= tol |phi|; S = Re phi^+ X; Y = Mpc X. Only the hopping blocks of Mpc
 * depend on the links:
 *   d(Mpc^+ Mpc) = dMpc^+ Mpc + Mpc^+ dMpc,  so  dS = -X^+ d(Mpc^+ Mpc) X = -2 Re Y^+ dMpc X,
 *   dMpc = -dMoe Mooee^-1 Meo - Moe Mooee^-1 dMeo = -(1/4)(dD_oe Mooee^-1 D_eo + D_oe Mooee^-1 dD_eo),
 * which gives dS = (1/2) Re B^+ dD A for the full fields
 *   A = Mooee^-1 D_eo X on even sites and X on odd sites,
 *   B = Mooee^-+ (D_oe)^+ Y on even sites and Y on odd sites   ((D_oe)^+ = the adjoint hop from odd to even).
 * Per link U_mu(x), with phase the boundary factor of the hop x -> x+mu, the functional
 * Re B^+ D A contains U_mu(x) through Re B(x)^+ (1 - gamma_mu) U A(x+mu) and through
 * Re B(x+mu)^+ (1 + gamma_mu) U^+ A(x), so with the colour outer products
 *   W1 = sum_{s,spin} A(x+mu) (x) [(1 - gamma_mu) B(x)]^+,   W2 = sum_{s,spin} A(x) (x) [(1 + gamma_mu) B(x+mu)]^+
 * its ambient gradient is phase (W1^+ + W2) and its su(3) force (U -> exp(eps T) U) is
 * TA(phase (-U W1 + W2 U^+)); S takes half of each:
 *   G = dS/dRe U + i dS/dIm U = (1/2) phase (W1^+ + W2),   F = (1/2) TA(phase (-U W1 + W2 U^+)).
 * X (odd sites) receives the solution; F and G may be NULL. Returns the number of CG iterations,
 * or -1 if maxiter was reached first; *S_out receives S.
 */
int dwf_oracle_pf_force(const int dims[4], int Ls, double M5, double mass, const int bc[4], const double* Ud,
                        const double* phid, double* Xd, double* Fd, double* Gd, double tol, int maxiter,
                        double* S_out, int nthreads) {
  const geom_t g = make_geom(dims, Ls, bc);
  const long n = g.V * Ls * 12;
  const cplx* phi = (const cplx*)phid;
  cplx* X = (cplx*)Xd;
  cplx* r = (cplx*)calloc(n, sizeof(cplx));
  cplx* p = (cplx*)calloc(n, sizeof(cplx));
  cplx* Ap = (cplx*)calloc(n, sizeof(cplx));
  cplx* A = (cplx*)calloc(n, sizeof(cplx));
  cplx* B = (cplx*)calloc(n, sizeof(cplx));
  cplx* t = (cplx*)calloc(n, sizeof(cplx));
  /* CG on Mpc^+ Mpc X = phi, odd sites */
  for (long i = 0; i < n; ++i) {
    X[i] = 0;
    r[i] = phi[i];
  }
  zero_parity(&g, r, 0);
  memcpy(p, r, sizeof(cplx) * n);
  const double phi_norm = sqrt(norm2(n, r));
  double rr = norm2(n, r);
  int k = 0;
  while (sqrt(rr) > tol * phi_norm) {
    if (k >= maxiter) {
      k = -1;
      break;
    }
    dwf_oracle_mdagm(dims, Ls, M5, mass, bc, Ud, (const double*)p, (double*)Ap, nthreads);
    const double alpha = rr / creal(inner(n, p, Ap));
    for (long i = 0; i < n; ++i) {
      X[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
    }
    const double rr_new = norm2(n, r);
    const double beta = rr_new / rr;
    rr = rr_new;
    for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    ++k;
  }
  *S_out = creal(inner(n, phi, X));
  /* A: X on odd sites, Mooee^-1 D_eo X on even sites */
  dwf_oracle_dhop(dims, Ls, bc, Ud, (const double*)X, (double*)t, 0, 0, nthreads);
  dwf_oracle_mooee(dims, Ls, M5, mass, (const double*)t, (double*)A, 0, 1, nthreads);
  /* B: Y = Mpc X on odd sites, Mooee^-+ (D_oe)^+ Y on even sites */
  dwf_oracle_mpc(dims, Ls, M5, mass, bc, Ud, (const double*)X, (double*)Ap, 0, nthreads);
  dwf_oracle_dhop(dims, Ls, bc, Ud, (const double*)Ap, (double*)t, 0, 1, nthreads);
  dwf_oracle_mooee(dims, Ls, M5, mass, (const double*)t, (double*)B, 1, 1, nthreads);
  for (long xs = 0; xs < g.V; ++xs) {
    int c[4];
    site_coords(&g, xs, c);
    if (site_parity(c) == 1)
      for (int i = 0; i < Ls * 12; ++i) {
        A[xs * Ls * 12 + i] = X[xs * Ls * 12 + i];
        B[xs * Ls * 12 + i] = Ap[xs * Ls * 12 + i];
      }
  }
  cplx gam[5][4][4];
  gamma_matrices(gam);
  const cplx* U = (const cplx*)Ud;
  cplx* F = (cplx*)Fd;
  cplx* G = (cplx*)Gd;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (long x = 0; x < g.V; ++x) {
    int c[4];
    site_coords(&g, x, c);
    for (int mu = 0; mu < 4; ++mu) {
      int cn[4] = {c[0], c[1], c[2], c[3]};
      cn[mu] = (c[mu] + 1) % g.L[mu];
      const long xf = lex_index(&g, cn);
      const double phase = c[mu] == g.L[mu] - 1 ? g.bc[mu] : 1.0;
      cplx W1[9] = {0}, W2[9] = {0};
      for (int s = 0; s < Ls; ++s) {
        const cplx* a_x = A + (x * Ls + s) * 12;
        const cplx* a_f = A + (xf * Ls + s) * 12;
        const cplx* b_x = B + (x * Ls + s) * 12;
        const cplx* b_f = B + (xf * Ls + s) * 12;
        cplx pb_x[12], pb_f[12]; /* (1 - gamma_mu) B(x), (1 + gamma_mu) B(x+mu) */
        for (int sp = 0; sp < 4; ++sp)
          for (int a = 0; a < 3; ++a) {
            cplx gx = 0, gf = 0;
            for (int sq = 0; sq < 4; ++sq) {
              gx += gam[mu][sp][sq] * b_x[sq * 3 + a];
              gf += gam[mu][sp][sq] * b_f[sq * 3 + a];
            }
            pb_x[sp * 3 + a] = b_x[sp * 3 + a] - gx;
            pb_f[sp * 3 + a] = b_f[sp * 3 + a] + gf;
          }
        for (int sp = 0; sp < 4; ++sp)
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              W1[a * 3 + b] += a_f[sp * 3 + a] * conj(pb_x[sp * 3 + b]);
              W2[a * 3 + b] += a_x[sp * 3 + a] * conj(pb_f[sp * 3 + b]);
            }
      }
      const cplx* u = U + (x * 4 + mu) * 9;
      if (F) {
        cplx Z[9], ta[9];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            cplx uW1 = 0, W2ud = 0;
            for (int q = 0; q < 3; ++q) {
              uW1 += u[a * 3 + q] * W1[q * 3 + b];
              W2ud += W2[a * 3 + q] * conj(u[b * 3 + q]);
            }
            Z[a * 3 + b] = phase * (-uW1 + W2ud);
          }
        traceless_antihermitian(Z, ta);
        for (int i = 0; i < 9; ++i) F[(x * 4 + mu) * 9 + i] = 0.5 * ta[i];
      }
      if (G)
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            G[(x * 4 + mu) * 9 + a * 3 + b] = 0.5 * phase * (conj(W1[b * 3 + a]) + W2[a * 3 + b]);
    }
  }
  free(r);
  free(p);
  free(Ap);
  free(A);
  free(B);
  free(t);
  return k;
}
