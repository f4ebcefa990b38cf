/*
 * CPU oracle for delayed approximate matrix assembly in multigrid
 * (Murray & Weinzierl, arXiv 2005.03606).  TEST INFRASTRUCTURE ONLY: the
 * tests, the smoke check and the benchmark's CPU-baseline leg call it; the
 * product path never does.  Plain FP64, written for readability, with no
 * blocking, fusion or reordering beyond the definitions it follows.  It
 * shares no code with the CUDA library.
 *
 * What it computes (each function cites the passage it follows):
 *   - eps(x) for the synthetic field families (Section "Results", Eq.
 *     "theta-setup" for the theta field; the others are plain definitions);
 *   - the element matrix A_c(s) of the weak form (Eq. "weak-form-of-
 *     assembly") with eps piecewise constant on an s^d sub-grid, eps taken at
 *     each sub-box centre (Section "Numerical computation of stencils");
 *     each sub-box integral of grad(phi_i).grad(phi_j) is done with the
 *     2-point Gauss rule per axis, which is exact for that polynomial;
 *   - adaptive per-cell accuracy: each cell walks the accuracy schedule and
 *     keeps the first matrix whose relative change in the element-wise
 *     maximum norm drops below C (Section "Adaptive stencil integration",
 *     Eq. "termination-criterion");
 *   - the hierarchical surplus A(s) - A(1) and its lossy storage
 *     (Section "Precision toggling and information density"), with the
 *     formats FP8-e4m3 / FP16 / FP32 plus a per-cell FP32 scale;
 *   - the paper's own truncated-float storage of that surplus (sign bit,
 *     truncated mantissa, signed-char exponent; p3 bytes per entry chosen
 *     against an absolute error threshold) and its compression factor;
 *   - d-linear 3:1 prolongation P, restriction R = P^T and element-local
 *     Ritz-Galerkin coarse operators R A P (Section "Rediscretisation and
 *     geometric projections"; Eq. for the Galerkin operator);
 *   - the additive cycles of Section "adaFAC-x" (plain additive multigrid,
 *     adaFAC-PI and adaFAC-Jac) with injection for adaFAC-PI;
 *   - damped Jacobi S = omega diag^-1(A) (Section "adaFAC-x"), the
 *     multiplicative V(nu1,nu2) cycle on the correction equation (Section
 *     "Multiplicative vs. additive schemes"), a dense solve on the coarsest
 *     grid and an outer residual-correction loop in FP64 with the relative
 *     residual stopping test (Section "Results": normalised residual).
 *
 * Index conventions: vertices of an N^d-cell grid are numbered
 * lexicographically on the (N+1)^d grid, x fastest; cells likewise on the
 * N^d grid; the 2^d local vertices of a cell are numbered by the bits
 * (b_x, b_y, b_z) of the local index.  Element matrices are stored full,
 * 2^d x 2^d row-major, cell after cell.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OC_CONST = 0, OC_DISC = 1, OC_FOURIER = 2, OC_BOXES = 3, OC_THETA = 4 };

/* Field parameters; the arrays are owned by the caller. */
typedef struct {
  int kind, dim, n_modes, n_boxes;
  double v_out, v_in;
  double center[3];
  double radius, sigma, theta, jump_x, jump_factor;
  const int32_t* k;      /* n_modes x 3 integer wavenumbers */
  const double* phase;   /* n_modes */
  const double* box_lo;  /* n_boxes x 3 */
  const double* box_hi;  /* n_boxes x 3 */
} oc_field;

static const double OC_PI = 3.14159265358979323846;

/* eps at point x (dim coordinates). */
double oc_eps(const oc_field* F, const double* x) {
  double e = F->v_out;
  int d = F->dim;
  if (F->kind == OC_DISC) {
    double r2 = 0.0;
    for (int a = 0; a < d; ++a) {
      double t = x[a] - F->center[a];
      r2 = r2 + t * t;
    }
    e = (r2 < F->radius * F->radius) ? F->v_in : F->v_out;
  } else if (F->kind == OC_FOURIER) {
    double g = 0.0;
    for (int m = 0; m < F->n_modes; ++m) {
      double kx = 0.0;
      for (int a = 0; a < d; ++a) kx += (double)F->k[3 * m + a] * x[a];
      g += cos(2.0 * OC_PI * kx + F->phase[m]);
    }
    e = F->v_out * exp(F->sigma * sqrt(2.0 / F->n_modes) * g);
  } else if (F->kind == OC_BOXES) {
    int inside = 0;
    for (int b = 0; b < F->n_boxes && !inside; ++b) {
      int in_b = 1;
      for (int a = 0; a < d; ++a)
        if (!(F->box_lo[3 * b + a] <= x[a] && x[a] < F->box_hi[3 * b + a])) in_b = 0;
      inside = in_b;
    }
    e = inside ? F->v_in : F->v_out;
  } else if (F->kind == OC_THETA) {
    double p = 1.0;
    for (int a = 0; a < d; ++a) p *= exp(-F->theta * x[a]) * cos(OC_PI * F->theta * x[a]);
    e = 1.0 + (0.3 / d) * p;
  }
  if (F->jump_factor != 1.0 && x[0] >= F->jump_x) e *= F->jump_factor;
  return e;
}

/* Sample coordinate of sub-box j (0 <= j < s) of cell i on an N-cell axis:
 * the sub-box centre (i + (j + 1/2)/s) / N, written as one exactly rounded
 * division of two integers. */
double oc_sample_coord(int N, int s, int i, int j) {
  return (double)(2 * ((int64_t)i * s + j) + 1) / (double)(2 * (int64_t)N * s);
}

/* 1D d-linear shape functions on [0,1] and their derivatives. */
static double shape1(int b, double t) { return b ? t : 1.0 - t; }
static double dshape1(int b) { return b ? 1.0 : -1.0; }

/*
 * Element matrix of cell `cell` (d integer coordinates) at accuracy s:
 *   A_ij = sum over sub-boxes q of eps(centre_q) * int_q grad phi_i . grad phi_j dx.
 * In reference coordinates xi in [0,1]^d (x = x0 + h xi) the integrand is
 * h^(d-2) grad_xi phi_i . grad_xi phi_j; each sub-box integral uses the
 * tensor 2-point Gauss rule.
 */
void oc_element_matrix(const oc_field* F, int N, const int* cell, int s, double* A) {
  const int d = F->dim, nv = 1 << d;
  const double h = 1.0 / N;
  const double g = 0.5 / sqrt(3.0);
  double hfac = 1.0;
  for (int a = 0; a < d - 2; ++a) hfac *= h;
  memset(A, 0, sizeof(double) * nv * nv);
  int nsub = 1;
  for (int a = 0; a < d; ++a) nsub *= s;
  const int ngp = nv;                     /* Gauss points per sub-box */
  double wq = 1.0;
  for (int a = 0; a < d; ++a) wq *= 0.5 / s;   /* 1D weight (1/s)/2 per axis */
  for (int q = 0; q < nsub; ++q) {
    int j[3] = {0, 0, 0};
    int rem = q;
    double x[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
      j[a] = rem % s;
      rem /= s;
      x[a] = oc_sample_coord(N, s, cell[a], j[a]);
    }
    const double e = oc_eps(F, x);
    for (int gp = 0; gp < ngp; ++gp) {
      double xi[3];
      for (int a = 0; a < d; ++a)
        xi[a] = (j[a] + 0.5 + (((gp >> a) & 1) ? g : -g)) / s;
      double grad[8][3];
      for (int i = 0; i < nv; ++i)
        for (int a = 0; a < d; ++a) {
          double v = dshape1((i >> a) & 1);
          for (int b = 0; b < d; ++b)
            if (b != a) v *= shape1((i >> b) & 1, xi[b]);
          grad[i][a] = v;
        }
      for (int i = 0; i < nv; ++i)
        for (int k = 0; k < nv; ++k) {
          double dot = 0.0;
          for (int a = 0; a < d; ++a) dot += grad[i][a] * grad[k][a];
          A[i * nv + k] += e * wq * dot;
        }
    }
  }
  for (int i = 0; i < nv * nv; ++i) A[i] *= hfac;
}

static int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  while (e-- > 0) r *= b;
  return r;
}

static void cell_coords(int d, int N, int64_t c, int* cc) {
  for (int a = 0; a < d; ++a) {
    cc[a] = (int)(c % N);
    c /= N;
  }
}

/* Element matrices of every cell of an N^d grid at accuracy s. */
void oc_assemble(const oc_field* F, int N, int s, double* A_all) {
  const int d = F->dim, nv = 1 << d;
  const int64_t ncell = ipow(N, d);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t c = 0; c < ncell; ++c) {
    int cc[3] = {0, 0, 0};
    cell_coords(d, N, c, cc);
    oc_element_matrix(F, N, cc, s, A_all + c * nv * nv);
  }
}

/* Element matrices of a list of cells (flat indices), for sampled checks. */
void oc_assemble_cells(const oc_field* F, int N, int s, const int64_t* cells, int64_t n,
                       double* A_out) {
  const int d = F->dim, nv = 1 << d;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < n; ++t) {
    int cc[3] = {0, 0, 0};
    cell_coords(d, N, cells[t], cc);
    oc_element_matrix(F, N, cc, s, A_out + t * nv * nv);
  }
}

/* Adaptive per-cell accuracy (Section "Adaptive stencil integration", Eq.
 * "termination-criterion"): each cell walks the accuracy schedule sched[0],
 * sched[1], ... and stops at the first level k >= 1 where the relative change
 * in the element-wise maximum norm,
 * ||A(sched[k]) - A(sched[k-1])||_max / ||A(sched[k-1])||_max, falls below C.
 * keep_old = 0: the cell stores A(sched[k]), the newest matrix (the rule's
 * text); keep_old = 1: it keeps A(sched[k-1]), the matrix that passed the
 * test (the Results' account of Table "memory-footprint": the lowest
 * accuracy approximation is used all the way through when the test finds no
 * difference).  s_cell receives the accuracy of the stored matrix. */
void oc_assemble_adaptive(const oc_field* F, int N, const int* sched, int n_s, double C, int keep_old,
                          double* A_all, int32_t* s_cell) {
  const int d = F->dim, nv = 1 << d;
  const int64_t ncell = ipow(N, d);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t c = 0; c < ncell; ++c) {
    int cc[3] = {0, 0, 0};
    cell_coords(d, N, c, cc);
    double* A = A_all + c * nv * nv;
    double Anew[64];
    oc_element_matrix(F, N, cc, sched[0], A);
    int sf = sched[0];
    for (int k = 1; k < n_s; ++k) {
      oc_element_matrix(F, N, cc, sched[k], Anew);
      double num = 0.0, den = 0.0;
      for (int i = 0; i < nv * nv; ++i) {
        if (fabs(Anew[i] - A[i]) > num) num = fabs(Anew[i] - A[i]);
        if (fabs(A[i]) > den) den = fabs(A[i]);
      }
      const int passed = num < C * den;
      if (passed && keep_old) break;   /* the older, lower-accuracy matrix stays */
      memcpy(A, Anew, sizeof(double) * nv * nv);
      sf = sched[k];
      if (passed) break;
    }
    s_cell[c] = sf;
  }
}

/* ---------------- lossy storage of the hierarchical surplus ---------------- */

/* Round x to the nearest value (ties to even) of a binary floating-point
 * format with `mbits` stored mantissa bits, minimum normal exponent `emin`
 * (subnormals below it) and largest finite value `maxval` (saturating). */
double oc_round_format(double x, int mbits, int emin, double maxval) {
  if (x == 0.0 || x != x) return x;
  double a = fabs(x);
  int E;
  frexp(a, &E);              /* a = f 2^E, f in [0.5, 1) => leading bit 2^(E-1) */
  int e = E - 1;
  if (e < emin) e = emin;
  double ulp = ldexp(1.0, e - mbits);
  double r = nearbyint(a / ulp) * ulp;   /* default rounding mode: to nearest even */
  if (r > maxval) r = maxval;
  return x < 0 ? -r : r;
}

double oc_round_e4m3(double x) { return oc_round_format(x, 3, -6, 448.0); }
double oc_round_f16(double x) { return oc_round_format(x, 10, -14, 65504.0); }

/*
 * Stored operator of the mixed-precision path for one cell.
 *   G   = eps_c32 * K, the geometric stencil with the cell-centre sample
 *         rounded to FP32 (the stored geometric part),
 *   D   = A - G (the hierarchical surplus, Section "Precision toggling"),
 *   Dm  = max |D_ij| over the off-diagonal entries i<j,
 *   An  = max |A_ij| over all entries, F = 2^d - 1.
 * Storage class: 0 (no payload; the paper's p3 = 0) if F*Dm <= tau*An;
 * 1 (FP8 e4m3, scale Dm/448)   if F*Dm*(16/448)   <= tau*An;
 * 2 (FP16, scale Dm/65504)     if F*Dm*(16/65504) <= tau*An;
 * 3 (FP32, no scale) otherwise.  The decoded surplus keeps symmetry and zero
 * row sums: only i<j entries are coded, the diagonal is minus the row sum.
 * Writes the decoded stored matrix At = G + decode(code(D)).
 */
int oc_compress_cell(int d, const double* A, double eps_c, const double* Kref, double tau,
                     double* At, double* scale_out) {
  const int nv = 1 << d;
  const double ec32 = (double)(float)eps_c;
  double Dm = 0.0, An = 0.0;
  double D[64];
  for (int i = 0; i < nv * nv; ++i) {
    D[i] = A[i] - ec32 * Kref[i];
    if (fabs(A[i]) > An) An = fabs(A[i]);
  }
  for (int i = 0; i < nv; ++i)
    for (int j = i + 1; j < nv; ++j)
      if (fabs(D[i * nv + j]) > Dm) Dm = fabs(D[i * nv + j]);
  const double F = nv - 1;
  int cls;
  if (F * Dm <= tau * An) cls = 0;
  else if (F * Dm * (16.0 / 448.0) <= tau * An) cls = 1;
  else if (F * Dm * (16.0 / 65504.0) <= tau * An) cls = 2;
  else cls = 3;
  double scale = 1.0;
  if (cls == 1) scale = (double)(float)(Dm / 448.0);
  if (cls == 2) scale = (double)(float)(Dm / 65504.0);
  double Dd[64];
  memset(Dd, 0, sizeof(Dd));
  for (int i = 0; i < nv; ++i)
    for (int j = i + 1; j < nv; ++j) {
      double v = D[i * nv + j], q = 0.0;
      if (cls == 1) q = oc_round_e4m3(v / scale) * scale;
      else if (cls == 2) q = oc_round_f16(v / scale) * scale;
      else if (cls == 3) q = (double)(float)v;
      Dd[i * nv + j] = q;
      Dd[j * nv + i] = q;
    }
  for (int i = 0; i < nv; ++i) {
    double rs = 0.0;
    for (int j = 0; j < nv; ++j)
      if (j != i) rs += Dd[i * nv + j];
    Dd[i * nv + i] = -rs;
  }
  for (int i = 0; i < nv * nv; ++i) At[i] = ec32 * Kref[i] + Dd[i];
  if (scale_out) *scale_out = scale;
  return cls;
}

/* Exact eps = 1 element matrix on an h-cell (the constant-eps precompute of
 * Section "Numerical computation of stencils"): one-sample assembly. */
void oc_kref(int d, int N, double* K) {
  oc_field one;
  memset(&one, 0, sizeof(one));
  one.kind = OC_CONST;
  one.dim = d;
  one.v_out = 1.0;
  one.jump_factor = 1.0;
  int cc[3] = {0, 0, 0};
  oc_element_matrix(&one, N, cc, 1, K);
}

/* Mixed-path stored operator for every cell: the FP64 A(s) in A_all is
 * replaced by the decoded stored matrices; classes go to cls. */
void oc_compress(const oc_field* F, int N, const double* A_all, double tau, double* At_all,
                 uint8_t* cls, double* scales) {
  const int d = F->dim, nv = 1 << d;
  const int64_t ncell = ipow(N, d);
  double K[64];
  oc_kref(d, N, K);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < ncell; ++c) {
    int cc[3] = {0, 0, 0};
    double x[3] = {0, 0, 0};
    cell_coords(d, N, c, cc);
    for (int a = 0; a < d; ++a) x[a] = oc_sample_coord(N, 1, cc[a], 0);
    double ec = oc_eps(F, x);
    double sc;
    cls[c] = (uint8_t)oc_compress_cell(d, A_all + c * nv * nv, ec, K, tau, At_all + c * nv * nv, &sc);
    if (scales) scales[c] = sc;
  }
}

/* ---------------- the paper's own storage format ----------------
 * Section "Precision toggling and information density": with p3 bytes per
 * entry (2 <= p3 < 8) an entry is a sign bit, m = 8 (p3 - 1) - 1 mantissa bits
 * and a plain signed-char exponent e^ in [-128, 127] without bias; the
 * mantissa is truncated, not rounded.  p3 = 8 is plain double precision and
 * p3 = 0 stores nothing (the entry decodes to zero).  Readings where the text
 * is silent: e^ = -128 is reserved for non-normalised values
 * (f / 2^m) 2^-127, which holds zero and anything below 2^-127; values at or
 * above 2^128 saturate to the largest encoding (2 - 2^-m) 2^127. */
double oc_pf_roundtrip(double x, int p3) {
  if (p3 >= 8) return x;
  if (p3 <= 0 || x == 0.0) return 0.0;
  const int m = 8 * (p3 - 1) - 1;
  const double a = fabs(x);
  int E;
  frexp(a, &E);            /* a = f 2^E with f in [0.5, 1): a in [2^(E-1), 2^E) */
  const int e = E - 1;
  double r;
  if (e > 127) {
    r = (2.0 - ldexp(1.0, -m)) * ldexp(1.0, 127);
  } else if (e >= -127) {
    const double frac = a / ldexp(1.0, e) - 1.0;               /* in [0, 1) */
    r = (1.0 + floor(ldexp(frac, m)) / ldexp(1.0, m)) * ldexp(1.0, e);
  } else {
    r = floor(ldexp(a, 127 + m)) * ldexp(1.0, -(127 + m));
  }
  return x < 0 ? -r : r;
}

/* Bytes per entry of one cell's hierarchical surplus (n entries): 0 when its
 * Frobenius norm is below the absolute threshold delta (the format would
 * store zeros), else the smallest p3 in 2..7 whose truncation error is at
 * most delta for every entry, else 8. */
int oc_pf_choose(const double* dA, int n, double delta) {
  double f2 = 0.0;
  for (int i = 0; i < n; ++i) f2 += dA[i] * dA[i];
  if (sqrt(f2) < delta) return 0;
  for (int p3 = 2; p3 <= 7; ++p3) {
    double err = 0.0;
    for (int i = 0; i < n; ++i) {
      const double e = fabs(dA[i] - oc_pf_roundtrip(dA[i], p3));
      if (e > err) err = e;
    }
    if (err <= delta) return p3;
  }
  return 8;
}

/* Every cell: surplus against the one-sample matrix eps_c[c] K (K = K_ref
 * h^(d-2), eps_c the cell-centre value the path stores), its p3, and the
 * decoded stored matrix eps_c K + roundtrip(A - eps_c K). */
void oc_paper_format(int d, int64_t ncell, const double* A_all, const double* eps_c, const double* K,
                     double delta, int32_t* p3_out, double* At_all) {
  const int nv = 1 << d, ne = nv * nv;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < ncell; ++c) {
    double dA[64];
    const double* A = A_all + c * ne;
    for (int i = 0; i < ne; ++i) dA[i] = A[i] - eps_c[c] * K[i];
    const int p3 = oc_pf_choose(dA, ne, delta);
    p3_out[c] = p3;
    if (At_all)
      for (int i = 0; i < ne; ++i) At_all[c * ne + i] = eps_c[c] * K[i] + oc_pf_roundtrip(dA[i], p3);
  }
}

/* ---------------- grid operators ---------------- */

static int64_t vidx(int d, int N, const int* v) {
  int64_t r = 0, m = 1;
  for (int a = 0; a < d; ++a) {
    r += v[a] * m;
    m *= (N + 1);
  }
  return r;
}

static int on_boundary(int d, int N, int64_t v) {
  for (int a = 0; a < d; ++a) {
    int64_t c = v % (N + 1);
    v /= (N + 1);
    if (c == 0 || c == N) return 1;
  }
  return 0;
}

/* y = A u with the Dirichlet rows removed (y = 0 on boundary vertices);
 * A is applied element by element (Eq. "weak-form-of-assembly"). */
void oc_apply(int d, int N, const double* A_all, const double* u, double* y) {
  const int nv = 1 << d;
  const int64_t nvert = ipow(N + 1, d), ncell = ipow(N, d);
  memset(y, 0, sizeof(double) * nvert);
  for (int64_t c = 0; c < ncell; ++c) {
    int cc[3] = {0, 0, 0};
    cell_coords(d, N, c, cc);
    int64_t gv[8];
    for (int i = 0; i < nv; ++i) {
      int v[3];
      for (int a = 0; a < d; ++a) v[a] = cc[a] + ((i >> a) & 1);
      gv[i] = vidx(d, N, v);
    }
    const double* A = A_all + c * nv * nv;
    for (int i = 0; i < nv; ++i) {
      double acc = 0.0;
      for (int j = 0; j < nv; ++j) acc += A[i * nv + j] * u[gv[j]];
      y[gv[i]] += acc;
    }
  }
  for (int64_t v = 0; v < nvert; ++v)
    if (on_boundary(d, N, v)) y[v] = 0.0;
}

/* Diagonal of the assembled operator (1 on boundary vertices, unused). */
void oc_diag(int d, int N, const double* A_all, double* diag) {
  const int nv = 1 << d;
  const int64_t nvert = ipow(N + 1, d), ncell = ipow(N, d);
  memset(diag, 0, sizeof(double) * nvert);
  for (int64_t c = 0; c < ncell; ++c) {
    int cc[3] = {0, 0, 0};
    cell_coords(d, N, c, cc);
    for (int i = 0; i < nv; ++i) {
      int v[3];
      for (int a = 0; a < d; ++a) v[a] = cc[a] + ((i >> a) & 1);
      diag[vidx(d, N, v)] += A_all[c * nv * nv + i * nv + i];
    }
  }
  for (int64_t v = 0; v < nvert; ++v)
    if (on_boundary(d, N, v)) diag[v] = 1.0;
}

/* r = b - A u on interior vertices, 0 on the boundary. */
void oc_residual(int d, int N, const double* A_all, const double* b, const double* u, double* r) {
  const int64_t nvert = ipow(N + 1, d);
  oc_apply(d, N, A_all, u, r);
  for (int64_t v = 0; v < nvert; ++v) r[v] = on_boundary(d, N, v) ? 0.0 : b[v] - r[v];
}

/* One damped Jacobi sweep u_out = u + omega diag^-1 (b - A u) (Section
 * "adaFAC-x": S = omega diag^-1(A)); every vertex uses the old u. */
void oc_jacobi(int d, int N, const double* A_all, const double* b, const double* u, double omega,
               double* u_out) {
  const int64_t nvert = ipow(N + 1, d);
  double* r = (double*)malloc(sizeof(double) * nvert);
  double* dg = (double*)malloc(sizeof(double) * nvert);
  oc_residual(d, N, A_all, b, u, r);
  oc_diag(d, N, A_all, dg);
  for (int64_t v = 0; v < nvert; ++v) u_out[v] = on_boundary(d, N, v) ? 0.0 : u[v] + omega * r[v] / dg[v];
  free(r);
  free(dg);
}

/* d-linear weight of coarse vertex offset `up` (0: left, 1: right) for the
 * fine vertex at fine index f on the 3:1 refined axis. */
static double pw(int f, int up) {
  int r = f % 3;
  double t = r / 3.0;
  return up ? t : 1.0 - t;
}

/* e_f += P e_c: d-linear interpolation from the Nc-cell grid to the 3Nc-cell grid. */
void oc_prolong_add(int d, int Nc, const double* ec, double* ef) {
  const int Nf = 3 * Nc;
  const int64_t nvf = ipow(Nf + 1, d);
  for (int64_t v = 0; v < nvf; ++v) {
    if (on_boundary(d, Nf, v)) continue;
    int fv[3] = {0, 0, 0};
    int64_t t = v;
    for (int a = 0; a < d; ++a) {
      fv[a] = (int)(t % (Nf + 1));
      t /= (Nf + 1);
    }
    double acc = 0.0;
    for (int corner = 0; corner < (1 << d); ++corner) {
      double w = 1.0;
      int cv[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) {
        int up = (corner >> a) & 1;
        w *= pw(fv[a], up);
        cv[a] = fv[a] / 3 + up;
        if (cv[a] > Nc) w = 0.0;
      }
      if (w != 0.0) acc += w * ec[vidx(d, Nc, cv)];
    }
    ef[v] += acc;
  }
}

/* b_c = P^T r_f (restriction as the transpose of prolongation), 0 on the coarse boundary. */
void oc_restrict(int d, int Nc, const double* rf, double* bc) {
  const int Nf = 3 * Nc;
  const int64_t nvf = ipow(Nf + 1, d), nvc = ipow(Nc + 1, d);
  memset(bc, 0, sizeof(double) * nvc);
  for (int64_t v = 0; v < nvf; ++v) {
    int fv[3] = {0, 0, 0};
    int64_t t = v;
    for (int a = 0; a < d; ++a) {
      fv[a] = (int)(t % (Nf + 1));
      t /= (Nf + 1);
    }
    for (int corner = 0; corner < (1 << d); ++corner) {
      double w = 1.0;
      int cv[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) {
        int up = (corner >> a) & 1;
        w *= pw(fv[a], up);
        cv[a] = fv[a] / 3 + up;
        if (cv[a] > Nc) w = 0.0;
      }
      if (w != 0.0) bc[vidx(d, Nc, cv)] += w * rf[v];
    }
  }
  for (int64_t v = 0; v < nvc; ++v)
    if (on_boundary(d, Nc, v)) bc[v] = 0.0;
}

/* Element-local Ritz-Galerkin coarse operator: for each coarse cell C,
 * A_C = sum over its 3^d children f of P_f^T A_f P_f, with P_f the d-linear
 * interpolation from C's vertices to f's vertices. */
void oc_galerkin(int d, int Nc, const double* A_fine, double* A_coarse) {
  const int nv = 1 << d, Nf = 3 * Nc;
  const int64_t ncc = ipow(Nc, d);
  int nchild = 1;
  for (int a = 0; a < d; ++a) nchild *= 3;
#pragma omp parallel for schedule(static)
  for (int64_t C = 0; C < ncc; ++C) {
    int cc[3] = {0, 0, 0};
    cell_coords(d, Nc, C, cc);
    double* AC = A_coarse + C * nv * nv;
    memset(AC, 0, sizeof(double) * nv * nv);
    for (int ch = 0; ch < nchild; ++ch) {
      int o[3] = {0, 0, 0}, rem = ch;
      for (int a = 0; a < d; ++a) {
        o[a] = rem % 3;
        rem /= 3;
      }
      int fc[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) fc[a] = 3 * cc[a] + o[a];
      int64_t f = 0, m = 1;
      for (int a = 0; a < d; ++a) {
        f += fc[a] * m;
        m *= Nf;
      }
      const double* Af = A_fine + f * nv * nv;
      double P[8][8];
      for (int i = 0; i < nv; ++i)
        for (int I = 0; I < nv; ++I) {
          double w = 1.0;
          for (int a = 0; a < d; ++a) {
            double t = (o[a] + ((i >> a) & 1)) / 3.0;
            w *= ((I >> a) & 1) ? t : 1.0 - t;
          }
          P[i][I] = w;
        }
      for (int I = 0; I < nv; ++I)
        for (int J = 0; J < nv; ++J) {
          double acc = 0.0;
          for (int i = 0; i < nv; ++i)
            for (int j = 0; j < nv; ++j) acc += P[i][I] * Af[i * nv + j] * P[j][J];
          AC[I * nv + J] += acc;
        }
    }
  }
}

/* ---------------- multigrid ---------------- */

typedef struct {
  int d, L;            /* levels 0 (coarsest, 3 cells/axis) .. L-1 (finest) */
  int N[16];
  double* A[16];       /* element matrices per level */
  double omega;
  int nu_pre, nu_post;
  double* dense;       /* coarsest interior system, factorised */
  int nint;
  int64_t* int_idx;
} oc_mg;

static double dot_interior(int d, int N, const double* a, const double* b) {
  const int64_t nvert = ipow(N + 1, d);
  double s = 0.0;
  for (int64_t v = 0; v < nvert; ++v)
    if (!on_boundary(d, N, v)) s += a[v] * b[v];
  return s;
}

/* Coarsest grid: dense FP64 Cholesky of the interior system. */
static void coarse_setup(oc_mg* mg) {
  const int d = mg->d, N = mg->N[0];
  const int64_t nvert = ipow(N + 1, d);
  int n = 0;
  mg->int_idx = (int64_t*)malloc(sizeof(int64_t) * nvert);
  for (int64_t v = 0; v < nvert; ++v)
    if (!on_boundary(d, N, v)) mg->int_idx[n++] = v;
  mg->nint = n;
  double* M = (double*)calloc((size_t)n * n, sizeof(double));
  double* e = (double*)calloc(nvert, sizeof(double));
  double* y = (double*)calloc(nvert, sizeof(double));
  for (int j = 0; j < n; ++j) {
    memset(e, 0, sizeof(double) * nvert);
    e[mg->int_idx[j]] = 1.0;
    oc_apply(d, N, mg->A[0], e, y);
    for (int i = 0; i < n; ++i) M[i * n + j] = y[mg->int_idx[i]];
  }
  /* Cholesky M = L L^T, L stored in the lower triangle */
  for (int j = 0; j < n; ++j) {
    double s = M[j * n + j];
    for (int k = 0; k < j; ++k) s -= M[j * n + k] * M[j * n + k];
    M[j * n + j] = sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = M[i * n + j];
      for (int k = 0; k < j; ++k) t -= M[i * n + k] * M[j * n + k];
      M[i * n + j] = t / M[j * n + j];
    }
  }
  mg->dense = M;
  free(e);
  free(y);
}

static void coarse_solve(const oc_mg* mg, const double* b, double* x) {
  const int n = mg->nint, d = mg->d, N = mg->N[0];
  const double* M = mg->dense;
  double* z = (double*)malloc(sizeof(double) * n);
  for (int i = 0; i < n; ++i) {
    double t = b[mg->int_idx[i]];
    for (int k = 0; k < i; ++k) t -= M[i * n + k] * z[k];
    z[i] = t / M[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = z[i];
    for (int k = i + 1; k < n; ++k) t -= M[k * n + i] * z[k];
    z[i] = t / M[i * n + i];
  }
  memset(x, 0, sizeof(double) * ipow(N + 1, d));
  for (int i = 0; i < n; ++i) x[mg->int_idx[i]] = z[i];
  free(z);
}

/* V(nu_pre, nu_post) cycle for A_l e = b starting from e = 0. */
static void vcycle(const oc_mg* mg, int l, const double* b, double* e) {
  const int d = mg->d, N = mg->N[l];
  const int64_t nvert = ipow(N + 1, d);
  if (l == 0) {
    coarse_solve(mg, b, e);
    return;
  }
  double* t = (double*)malloc(sizeof(double) * nvert);
  memset(e, 0, sizeof(double) * nvert);
  for (int k = 0; k < mg->nu_pre; ++k) {
    oc_jacobi(d, N, mg->A[l], b, e, mg->omega, t);
    memcpy(e, t, sizeof(double) * nvert);
  }
  double* r = (double*)malloc(sizeof(double) * nvert);
  oc_residual(d, N, mg->A[l], b, e, r);
  const int Nc = mg->N[l - 1];
  const int64_t nvc = ipow(Nc + 1, d);
  double* bc = (double*)malloc(sizeof(double) * nvc);
  double* ecv = (double*)malloc(sizeof(double) * nvc);
  oc_restrict(d, Nc, r, bc);
  vcycle(mg, l - 1, bc, ecv);
  oc_prolong_add(d, Nc, ecv, e);
  for (int k = 0; k < mg->nu_post; ++k) {
    oc_jacobi(d, N, mg->A[l], b, e, mg->omega, t);
    memcpy(e, t, sizeof(double) * nvert);
  }
  free(t);
  free(r);
  free(bc);
  free(ecv);
}

/*
 * Solve A u = f with f_v = f_const * h^d (the load vector of a constant
 * right-hand side), u = u0 on entry (0 if u0 is NULL).  The V-cycle acts on
 * the residual equation; the outer FP64 loop is either
 *   outer = 0: residual correction (iterative refinement)
 *              r = f - A u;  e = V(r);  u += e,
 *   outer = 1: flexible conjugate gradients (Notay's FCG(1)) with the
 *              V-cycle as preconditioner:  z = V(r); p = z - (z.q_old /
 *              p_old.q_old) p_old;  q = A p;  alpha = p.r / p.q;
 *              u += alpha p;  r -= alpha q.
 * It stops when ||r||_2 <= rtol ||f||_2 on the interior vertices (||r_0||
 * in place of ||f|| when f = 0, the paper's normalised residual) or after
 * max_cycles V-cycles.  A_fine holds the finest element matrices; coarse
 * levels are built by element-local Galerkin products down to 3 cells per
 * axis.  history[k] = ||r_k|| / ||f|| for k = 0..cycles; the last entry is
 * the true residual f - A u recomputed at the end.
 * Returns the number of cycles, or -1 on bad input.
 */
int oc_solve(int d, int N, const double* A_fine, double f_const, const double* u0, double omega,
             int nu_pre, int nu_post, double rtol, int max_cycles, int outer, double* u_out,
             double* history) {
  oc_mg mg;
  memset(&mg, 0, sizeof(mg));
  mg.d = d;
  mg.omega = omega;
  mg.nu_pre = nu_pre;
  mg.nu_post = nu_post;
  int L = 0, n = N;
  while (n >= 3) {
    L++;
    if (n == 3) break;
    if (n % 3) return -1;
    n /= 3;
  }
  if (n != 3) return -1;
  mg.L = L;
  const int nv = 1 << d;
  n = N;
  for (int l = L - 1; l >= 0; --l) {
    mg.N[l] = n;
    n /= 3;
  }
  mg.A[L - 1] = (double*)A_fine;
  for (int l = L - 2; l >= 0; --l) {
    mg.A[l] = (double*)malloc(sizeof(double) * ipow(mg.N[l], d) * nv * nv);
    oc_galerkin(d, mg.N[l], mg.A[l + 1], mg.A[l]);
  }
  coarse_setup(&mg);
  const int64_t nvert = ipow(N + 1, d);
  double h = 1.0 / N, hd = 1.0;
  for (int a = 0; a < d; ++a) hd *= h;
  double* f = (double*)malloc(sizeof(double) * nvert);
  double* r = (double*)malloc(sizeof(double) * nvert);
  double* e = (double*)malloc(sizeof(double) * nvert);
  double* p = (double*)calloc(nvert, sizeof(double));
  double* q = (double*)calloc(nvert, sizeof(double));
  for (int64_t v = 0; v < nvert; ++v) {
    f[v] = on_boundary(d, N, v) ? 0.0 : f_const * hd;
    u_out[v] = (u0 && !on_boundary(d, N, v)) ? u0[v] : 0.0;
  }
  oc_residual(d, N, mg.A[L - 1], f, u_out, r);
  double fn = sqrt(dot_interior(d, N, f, f));
  double rn = sqrt(dot_interior(d, N, r, r));
  double ref = fn > 0 ? fn : rn;
  if (ref == 0) ref = 1;
  int k = 0;
  if (history) history[0] = rn / ref;
  double pq = 0.0;
  while (rn > rtol * ref && k < max_cycles) {
    vcycle(&mg, L - 1, r, e);               /* e = z = V(r) */
    if (outer == 0) {
      for (int64_t v = 0; v < nvert; ++v) u_out[v] += e[v];
      oc_residual(d, N, mg.A[L - 1], f, u_out, r);
    } else {
      if (k == 0) {
        memcpy(p, e, sizeof(double) * nvert);
      } else {
        double beta = -dot_interior(d, N, e, q) / pq;
        for (int64_t v = 0; v < nvert; ++v) p[v] = e[v] + beta * p[v];
      }
      oc_apply(d, N, mg.A[L - 1], p, q);
      pq = dot_interior(d, N, p, q);
      double alpha = dot_interior(d, N, p, r) / pq;
      for (int64_t v = 0; v < nvert; ++v) {
        u_out[v] += alpha * p[v];
        r[v] -= alpha * q[v];
      }
    }
    rn = sqrt(dot_interior(d, N, r, r));
    ++k;
    if (history) history[k] = rn / ref;
  }
  oc_residual(d, N, mg.A[L - 1], f, u_out, r);
  if (history) history[k] = sqrt(dot_interior(d, N, r, r)) / ref;
  for (int l = L - 2; l >= 0; --l) free(mg.A[l]);
  free(mg.dense);
  free(mg.int_idx);
  free(f);
  free(r);
  free(e);
  free(p);
  free(q);
  return k;
}

/* One V-cycle on level data given explicitly (for step-by-step checks):
 * e = V(b) on the finest level of the hierarchy built from A_fine. */
int oc_vcycle_once(int d, int N, const double* A_fine, const double* b, double omega, int nu_pre,
                   int nu_post, double* e) {
  oc_mg mg;
  memset(&mg, 0, sizeof(mg));
  mg.d = d;
  mg.omega = omega;
  mg.nu_pre = nu_pre;
  mg.nu_post = nu_post;
  int L = 0, n = N;
  while (n >= 3) {
    L++;
    if (n == 3) break;
    if (n % 3) return -1;
    n /= 3;
  }
  if (n != 3) return -1;
  mg.L = L;
  const int nv = 1 << d;
  n = N;
  for (int l = L - 1; l >= 0; --l) {
    mg.N[l] = n;
    n /= 3;
  }
  mg.A[L - 1] = (double*)A_fine;
  for (int l = L - 2; l >= 0; --l) {
    mg.A[l] = (double*)malloc(sizeof(double) * ipow(mg.N[l], d) * nv * nv);
    oc_galerkin(d, mg.N[l], mg.A[l + 1], mg.A[l]);
  }
  coarse_setup(&mg);
  vcycle(&mg, L - 1, b, e);
  for (int l = L - 2; l >= 0; --l) free(mg.A[l]);
  free(mg.dense);
  free(mg.int_idx);
  return 0;
}

/* Injection of fine vertex values to the coinciding coarse vertices (the
 * restriction of adaFAC-PI's auxiliary equation, Section "adaFAC-x"). */
void oc_inject(int d, int Nc, const double* rf, double* bc) {
  const int Nf = 3 * Nc;
  const int64_t ncv = ipow(Nc + 1, d);
  for (int64_t v = 0; v < ncv; ++v) {
    int c[3] = {0, 0, 0};
    int64_t t = v;
    for (int a = 0; a < d; ++a) {
      c[a] = (int)(t % (Nc + 1));
      t /= Nc + 1;
    }
    int f[3] = {3 * c[0], 3 * c[1], 3 * c[2]};
    bc[v] = on_boundary(d, Nc, v) ? 0.0 : rf[vidx(d, Nf, f)];
  }
}

/* One additive cycle for the correction equation A e = b, from e = 0
 * (Section "adaFAC-x", Eq. "adaFAC-x", in correction form): the fine residual
 * is restricted to every level; every level but the coarsest takes one
 * damped Jacobi step on it, c_l = omega D_l^-1 r_l, the coarsest is solved
 * exactly, and all corrections are prolongated to the finest level and
 * added.  variants 1 (adaFAC-PI) and 2 (adaFAC-Jac) damp each c_l (l above
 * the coarsest) with an auxiliary Jacobi step on the next coarser level,
 * s = omega D_(l-1)^-1 t, which mimics the overshoot of the coarse
 * corrections running concurrently:
 *   adaFAC-PI:  t = I r_l (injection), c_l = S_l r_l - P s (the BPX-like pair
 *               P, I);
 *   adaFAC-Jac: t = R (r_l - A_l S_l r_l), the restriction by the transpose of
 *               the Jacobi-smoothed prolongation (I - S_l A_l) P, and the
 *               auxiliary correction is taken out through the level's own
 *               smoother, c_l = S_l (r_l - A_l P s), the form of the AFACx
 *               schemes that adaFAC-x derives from (P~ = S_l A_l P).
 * variant 0 is plain additive multigrid.  Levels of mg: 0 coarsest .. L-1
 * finest. */
static void additive_cycle(const oc_mg* mg, const double* b, double* e, int variant) {
  const int d = mg->d, L = mg->L;
  double* r[16];
  double* c[16];
  for (int l = 0; l < L; ++l) {
    const int64_t nv = ipow(mg->N[l] + 1, d);
    r[l] = (double*)calloc(nv, sizeof(double));
    c[l] = (double*)calloc(nv, sizeof(double));
  }
  memcpy(r[L - 1], b, sizeof(double) * ipow(mg->N[L - 1] + 1, d));
  for (int l = L - 1; l >= 1; --l) oc_restrict(d, mg->N[l - 1], r[l], r[l - 1]);
  coarse_solve(mg, r[0], c[0]);
  for (int l = 1; l < L; ++l) {
    const int N = mg->N[l], Nc = mg->N[l - 1];
    const int64_t nv = ipow(N + 1, d), ncv = ipow(Nc + 1, d);
    double* zero = (double*)calloc(nv, sizeof(double));
    oc_jacobi(d, N, mg->A[l], r[l], zero, mg->omega, c[l]);
    if (variant == 1 || variant == 2) {
      double* t = (double*)calloc(ncv, sizeof(double));
      double* sc = (double*)calloc(ncv, sizeof(double));
      double* zc = (double*)calloc(ncv, sizeof(double));
      if (variant == 1) {
        oc_inject(d, Nc, r[l], t);
      } else {
        double* q = (double*)calloc(nv, sizeof(double));
        oc_residual(d, N, mg->A[l], r[l], c[l], q);
        oc_restrict(d, Nc, q, t);
        free(q);
      }
      oc_jacobi(d, Nc, mg->A[l - 1], t, zc, mg->omega, sc);
      if (variant == 1) {
        for (int64_t v = 0; v < ncv; ++v) sc[v] = -sc[v];
        oc_prolong_add(d, Nc, sc, c[l]);
      } else {
        /* c_l = S_l (r_l - A_l y), y = P s: one Jacobi step from y, minus y */
        double* y = (double*)calloc(nv, sizeof(double));
        oc_prolong_add(d, Nc, sc, y);
        oc_jacobi(d, N, mg->A[l], r[l], y, mg->omega, c[l]);
        for (int64_t v = 0; v < nv; ++v) c[l][v] -= y[v];
        free(y);
      }
      free(t);
      free(sc);
      free(zc);
    }
    free(zero);
  }
  for (int l = 1; l < L; ++l) oc_prolong_add(d, mg->N[l - 1], c[l - 1], c[l]);
  memcpy(e, c[L - 1], sizeof(double) * ipow(mg->N[L - 1] + 1, d));
  for (int l = 0; l < L; ++l) {
    free(r[l]);
    free(c[l]);
  }
}

int oc_additive_once(int d, int N, const double* A_fine, const double* b, double omega, int variant, double* e) {
  oc_mg mg;
  memset(&mg, 0, sizeof(mg));
  mg.d = d;
  mg.omega = omega;
  int L = 0, n = N;
  while (n >= 3) {
    L++;
    if (n == 3) break;
    if (n % 3) return -1;
    n /= 3;
  }
  if (n != 3) return -1;
  mg.L = L;
  const int nv = 1 << d;
  n = N;
  for (int l = L - 1; l >= 0; --l) {
    mg.N[l] = n;
    n /= 3;
  }
  mg.A[L - 1] = (double*)A_fine;
  for (int l = L - 2; l >= 0; --l) {
    mg.A[l] = (double*)malloc(sizeof(double) * ipow(mg.N[l], d) * nv * nv);
    oc_galerkin(d, mg.N[l], mg.A[l + 1], mg.A[l]);
  }
  coarse_setup(&mg);
  additive_cycle(&mg, b, e, variant);
  for (int l = L - 2; l >= 0; --l) free(mg.A[l]);
  free(mg.dense);
  free(mg.int_idx);
  return 0;
}

int oc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
