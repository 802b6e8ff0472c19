/* oracle.c -- plain CPU FP64 restatement of the non-singular boundary integral method
 * (Klaseboer, Sepehrirahnama & Chan, arXiv 1706.07919).  TEST INFRASTRUCTURE ONLY: see oracle.h.
 *
 * Written for a reader checking it against the paper: no blocking, no fusion, no reordering.
 * OpenMP only splits independent rows / points / output samples across threads.
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;
static const double PI = 3.14159265358979323846264338327950288;

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------------------------
 * Quadrature (Sec. 3: ordinary Gauss quadrature suffices once the kernels are regular).  The paper names no rule; the
 * reading used here is a collapsed-coordinate tensor Gauss-Legendre rule.
 * ------------------------------------------------------------------------------------------ */
int or_gauss_legendre01(int n, double* x, double* w) {
  if (n < 1 || n > 64) return -1;
  for (int i = 0; i < n; ++i) {
    /* Root i of P_n on [-1, 1], by Newton from the Chebyshev-like first guess. */
    double z = cos(PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p_prev = 0.0, p = 1.0;
      for (int j = 1; j <= n; ++j) {          /* Bonnet recurrence for P_j(z) */
        double p_next = ((2.0 * j - 1.0) * z * p - (j - 1.0) * p_prev) / j;
        p_prev = p;
        p = p_next;
      }
      dp = n * (z * p - p_prev) / (z * z - 1.0); /* P_n'(z) */
      double dz = p / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    {
      double p_prev = 0.0, p = 1.0;
      for (int j = 1; j <= n; ++j) {
        double p_next = ((2.0 * j - 1.0) * z * p - (j - 1.0) * p_prev) / j;
        p_prev = p;
        p = p_next;
      }
      dp = n * (z * p - p_prev) / (z * z - 1.0);
    }
    /* map [-1, 1] -> [0, 1] by t = (1 - z)/2; z decreases with i, so t ascends */
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp); /* (2/((1-z^2) P_n'^2)) / 2 */
  }
  return 0;
}

void or_shape6(double xi, double eta, double* N, double* dNxi, double* dNeta) {
  /* Quadratic Lagrange interpolants on the 6-node triangle (Sec. 3: quadratic elements and
   * quadratic interpolation).  Barycentric L1 = 1 - xi - eta, L2 = xi, L3 = eta. */
  double L1 = 1.0 - xi - eta, L2 = xi, L3 = eta;
  N[0] = L1 * (2.0 * L1 - 1.0);
  N[1] = L2 * (2.0 * L2 - 1.0);
  N[2] = L3 * (2.0 * L3 - 1.0);
  N[3] = 4.0 * L1 * L2;
  N[4] = 4.0 * L2 * L3;
  N[5] = 4.0 * L3 * L1;
  if (dNxi) {
    /* d/dxi: dL1 = -1, dL2 = 1, dL3 = 0 */
    dNxi[0] = -(4.0 * L1 - 1.0);
    dNxi[1] = 4.0 * L2 - 1.0;
    dNxi[2] = 0.0;
    dNxi[3] = 4.0 * (L1 - L2);
    dNxi[4] = 4.0 * L3;
    dNxi[5] = -4.0 * L3;
  }
  if (dNeta) {
    /* d/deta: dL1 = -1, dL2 = 0, dL3 = 1 */
    dNeta[0] = -(4.0 * L1 - 1.0);
    dNeta[1] = 0.0;
    dNeta[2] = 4.0 * L3 - 1.0;
    dNeta[3] = -4.0 * L2;
    dNeta[4] = 4.0 * L2;
    dNeta[5] = 4.0 * (L1 - L3);
  }
}

void or_shape3(double xi, double eta, double* N, double* dNxi, double* dNeta) {
  /* Linear interpolants on the 3-node triangle (Sec. 4: the cross-check with linear elements and
   * linear interpolation): the barycentric coordinates themselves. */
  N[0] = 1.0 - xi - eta;
  N[1] = xi;
  N[2] = eta;
  if (dNxi) { dNxi[0] = -1.0; dNxi[1] = 1.0; dNxi[2] = 0.0; }
  if (dNeta) { dNeta[0] = -1.0; dNeta[1] = 0.0; dNeta[2] = 1.0; }
}

/* Shape functions of an element with np = 6 (quadratic) or np = 3 (linear) nodes. */
static void shape_n(int np, double xi, double eta, double* N, double* dNxi, double* dNeta) {
  if (np == 3) or_shape3(xi, eta, N, dNxi, dNeta);
  else or_shape6(xi, eta, N, dNxi, dNeta);
}

/* Reference coordinates of the six local nodes. */
static const double REF_NODE[6][2] = {{0, 0}, {1, 0}, {0, 1}, {0.5, 0}, {0.5, 0.5}, {0, 0.5}};

/* n*n Duffy points of the sub-triangle (V, A, B) collapsed onto V:
 * p = V + u (A - V) + u v (B - A), dA = u |det(A - V, B - A)| du dv. */
static int duffy(int n, const double* gx, const double* gw, const double V[2], const double A[2],
                 const double B[2], double* xi, double* eta, double* w) {
  double e1[2] = {A[0] - V[0], A[1] - V[1]}, e2[2] = {B[0] - A[0], B[1] - A[1]};
  double det = fabs(e1[0] * e2[1] - e1[1] * e2[0]);
  int c = 0;
  for (int iu = 0; iu < n; ++iu)
    for (int iv = 0; iv < n; ++iv) {
      double u = gx[iu], v = gx[iv];
      xi[c] = V[0] + u * e1[0] + u * v * e2[0];
      eta[c] = V[1] + u * e1[1] + u * v * e2[1];
      w[c] = gw[iu] * gw[iv] * u * det;
      ++c;
    }
  return c;
}

int or_rule_std(int n, double* xi, double* eta, double* w) {
  double gx[64], gw[64];
  if (or_gauss_legendre01(n, gx, gw)) return -1;
  return duffy(n, gx, gw, REF_NODE[0], REF_NODE[1], REF_NODE[2], xi, eta, w);
}

int or_rule_near(int n, int a, double* xi, double* eta, double* w) {
  double gx[64], gw[64];
  if (a < 0 || a > 5 || or_gauss_legendre01(n, gx, gw)) return -1;
  if (a < 3) { /* vertex node: one triangle collapsed onto it */
    return duffy(n, gx, gw, REF_NODE[a], REF_NODE[(a + 1) % 3], REF_NODE[(a + 2) % 3], xi, eta, w);
  }
  /* mid-edge node on edge (pa, pb), opposite vertex pc: sub-triangles (M,pb,pc), (M,pc,pa) */
  int pa = a - 3, pb = (a - 2) % 3, pc = (a - 1) % 3;
  int c = duffy(n, gx, gw, REF_NODE[a], REF_NODE[pb], REF_NODE[pc], xi, eta, w);
  c += duffy(n, gx, gw, REF_NODE[a], REF_NODE[pc], REF_NODE[pa], xi + c, eta + c, w + c);
  return c;
}

/* Isoparametric geometry of an element with np nodes at (xi, eta): position, unit normal
 * t1 x t2 / J, J, and the np shape values. */
static void elem_point(const double* nodes, const int32_t* el, int np, double xi, double eta, double x[3],
                       double nu[3], double* J, double Nv[6]) {
  double dx[6], de[6];
  shape_n(np, xi, eta, Nv, dx, de);
  double t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0};
  x[0] = x[1] = x[2] = 0.0;
  for (int a = 0; a < np; ++a) {
    const double* X = nodes + 3 * (int64_t)el[a];
    for (int d = 0; d < 3; ++d) {
      x[d] += Nv[a] * X[d];
      t1[d] += dx[a] * X[d];
      t2[d] += de[a] * X[d];
    }
  }
  double n[3] = {t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2],
                 t1[0] * t2[1] - t1[1] * t2[0]};
  *J = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (int d = 0; d < 3; ++d) nu[d] = n[d] / *J;
}

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------------------------------
 * Eq. BRIEF assembly (Sec. 3, App. A): every node x_i is a collocation point.
 * ------------------------------------------------------------------------------------------ */
/* The rules of one assembly: standard points, and near points per local node. */
typedef struct {
  int nstd;
  double sxi[256], seta[256], sw[256];
  int nnear[6];
  double nxi[6][512], neta[6][512], nw[6][512];
} rules_t;

static void make_rules(int ng, int ng_near, rules_t* r) {
  r->nstd = or_rule_std(ng, r->sxi, r->seta, r->sw);
  for (int a = 0; a < 6; ++a) r->nnear[a] = or_rule_near(ng_near, a, r->nxi[a], r->neta[a], r->nw[a]);
}

/* Row i: Hrow[j], Gmrow[j] (accumulated) and alpha_i, beta_i. */
static void row_integrals(const double* nodes, int64_t N, const int32_t* elems, int np, int64_t E,
                          const double* normals, double k, const rules_t* ru, int64_t i, cplx* Hrow,
                          cplx* Gmrow, cplx* alpha_i, cplx* beta_i) {
  (void)N;
  const double* xi0 = nodes + 3 * i;   /* collocation point x_i */
  const double* nu0 = normals + 3 * i; /* its normal nu_i */
  cplx al = 0.0, be = 0.0;
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* el = elems + (int64_t)np * e;
    int own = -1; /* local index of node i in element e, if any (a vertex for np = 3) */
    for (int a = 0; a < np; ++a)
      if (el[a] == i) own = a;
    const double *qx = ru->sxi, *qe = ru->seta, *qw = ru->sw;
    int nq = ru->nstd;
    if (own >= 0) {
      qx = ru->nxi[own];
      qe = ru->neta[own];
      qw = ru->nw[own];
      nq = ru->nnear[own];
    }
    for (int q = 0; q < nq; ++q) {
      double x[3], nu[3], J, Nv[6];
      elem_point(nodes, el, np, qx[q], qe[q], x, nu, &J, Nv);
      double r[3] = {x[0] - xi0[0], x[1] - xi0[1], x[2] - xi0[2]};
      double R = sqrt(dot3(r, r));
      cplx eikr = cexp(I * k * R);
      cplx G = eikr / R;                                           /* Eq. Green_func */
      cplx dG = eikr * (I * k * R - 1.0) * dot3(r, nu) / (R * R * R); /* dG/dnu at x */
      double s = k * dot3(nu0, r);
      /* Eqs. g_function, f_function; at k = 0 (the zero-frequency term of Eq. inverseFourier) f
       * takes its limit sin(k nu_i.r)/k -> nu_i.r, while g -> 1 and G -> 1/R need no change */
      double g = cos(s), f = (k == 0.0) ? dot3(nu0, r) : sin(s) / k;
      double dg = -k * sin(s) * dot3(nu0, nu), df = cos(s) * dot3(nu0, nu);
      double wJ = qw[q] * J;
      for (int a = 0; a < np; ++a) {
        Hrow[el[a]] += wJ * Nv[a] * dG;
        Gmrow[el[a]] += wJ * Nv[a] * G;
      }
      al += wJ * (g * dG - dg * G);
      be += wJ * (f * dG - df * G);
    }
  }
  *alpha_i = al;
  *beta_i = be;
}

static int check_mesh(int64_t N, const int32_t* elems, int np, int64_t E, double k, int ng, int ng_near) {
  if (N < 1 || E < 1 || !(k >= 0.0) || ng < 1 || ng > 16 || ng_near < 1 || ng_near > 16) return -1;
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < np; ++a)
      if (elems[np * e + a] < 0 || elems[np * e + a] >= N) return -1;
  return 0;
}

static int assemble_raw_n(const double* nodes, int64_t N, const int32_t* elems, int np, int64_t E,
                          const double* normals, double k, int ng, int ng_near, cplx* H, cplx* Gm,
                          cplx* alpha, cplx* beta) {
  if (check_mesh(N, elems, np, E, k, ng, ng_near)) return -1;
  rules_t* ru = (rules_t*)malloc(sizeof(rules_t));
  if (!ru) return -3;
  make_rules(ng, ng_near, ru);
  memset(H, 0, sizeof(cplx) * N * N);
  memset(Gm, 0, sizeof(cplx) * N * N);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < N; ++i)
    row_integrals(nodes, N, elems, np, E, normals, k, ru, i, H + i * N, Gm + i * N, alpha + i, beta + i);
  free(ru);
  return 0;
}

/* Rows rows[0..nrows) of the system of or_assemble_system: A_rows [nrows][N], b_rows [nrows]. */
static int assemble_rows_n(const double* nodes, int64_t N, const int32_t* elems, int np, int64_t E,
                           const double* normals, const uint8_t* bc, double k, const double* dir, int ng,
                           int ng_near, const int64_t* rows, int64_t nrows, cplx* A_rows, cplx* b_rows) {
  if (check_mesh(N, elems, np, E, k, ng, ng_near)) return -1;
  for (int64_t t = 0; t < nrows; ++t)
    if (rows[t] < 0 || rows[t] >= N) return -1;
  rules_t* ru = (rules_t*)malloc(sizeof(rules_t));
  cplx* known = (cplx*)malloc(sizeof(cplx) * N);
  if (!ru || !known) {
    free(ru); free(known);
    return -3;
  }
  make_rules(ng, ng_near, ru);
  for (int64_t j = 0; j < N; ++j) {
    cplx pinc = cexp(I * k * dot3(dir, nodes + 3 * j));
    known[j] = bc[j] ? -pinc : -(I * k * dot3(dir, normals + 3 * j)) * pinc;
  }
  int rc = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < nrows; ++t) {
    const int64_t i = rows[t];
    cplx* H = (cplx*)calloc(N, sizeof(cplx));
    cplx* Gm = (cplx*)calloc(N, sizeof(cplx));
    if (!H || !Gm) {
      rc = -3;
    } else {
      cplx al, be;
      row_integrals(nodes, N, elems, np, E, normals, k, ru, i, H, Gm, &al, &be);
      cplx bi = 0.0;
      for (int64_t j = 0; j < N; ++j) {
        cplx C = H[j] - (i == j ? 4.0 * PI + al : 0.0); /* multiplies P_j  */
        cplx D = -(Gm[j] + (i == j ? be : 0.0));        /* multiplies P'_j */
        if (bc[j] == 0) {
          A_rows[t * N + j] = C;
          bi -= D * known[j];
        } else {
          A_rows[t * N + j] = D;
          bi -= C * known[j];
        }
      }
      b_rows[t] = bi;
    }
    free(H);
    free(Gm);
  }
  free(ru);
  free(known);
  return rc;
}

static int assemble_system_n(const double* nodes, int64_t N, const int32_t* elems, int np, int64_t E,
                             const double* normals, const uint8_t* bc, double k, const double* dir,
                             int ng, int ng_near, cplx* A, cplx* b) {
  cplx* H = (cplx*)malloc(sizeof(cplx) * N * N);
  cplx* Gm = (cplx*)malloc(sizeof(cplx) * N * N);
  cplx* al = (cplx*)malloc(sizeof(cplx) * N);
  cplx* be = (cplx*)malloc(sizeof(cplx) * N);
  cplx* known = (cplx*)malloc(sizeof(cplx) * N);
  if (!H || !Gm || !al || !be || !known) {
    free(H); free(Gm); free(al); free(be); free(known);
    return -3;
  }
  int rc = assemble_raw_n(nodes, N, elems, np, E, normals, k, ng, ng_near, H, Gm, al, be);
  if (rc == 0) {
    /* Known boundary values of the scattered field (Sec. 4): soft p_scat = -p_inc,
     * hard dp_scat/dn = -dp_inc/dn, for the unit plane wave p_inc = exp(i k d.x). */
    for (int64_t j = 0; j < N; ++j) {
      cplx pinc = cexp(I * k * dot3(dir, nodes + 3 * j));
      known[j] = bc[j] ? -pinc : -(I * k * dot3(dir, normals + 3 * j)) * pinc;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
      cplx bi = 0.0;
      for (int64_t j = 0; j < N; ++j) {
        cplx C = H[i * N + j] - (i == j ? 4.0 * PI + al[i] : 0.0); /* multiplies P_j  */
        cplx D = -(Gm[i * N + j] + (i == j ? be[i] : 0.0));        /* multiplies P'_j */
        if (bc[j] == 0) {
          A[i * N + j] = C;
          bi -= D * known[j];
        } else {
          A[i * N + j] = D;
          bi -= C * known[j];
        }
      }
      b[i] = bi;
    }
  }
  free(H); free(Gm); free(al); free(be); free(known);
  return rc;
}

int or_assemble_raw(const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                    const double* normals, double k, int ng, int ng_near, cplx* H, cplx* Gm,
                    cplx* alpha, cplx* beta) {
  return assemble_raw_n(nodes, N, elems, 6, E, normals, k, ng, ng_near, H, Gm, alpha, beta);
}
int or_assemble_rows(const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                     const double* normals, const uint8_t* bc, double k, const double* dir, int ng,
                     int ng_near, const int64_t* rows, int64_t nrows, cplx* A_rows, cplx* b_rows) {
  return assemble_rows_n(nodes, N, elems, 6, E, normals, bc, k, dir, ng, ng_near, rows, nrows, A_rows, b_rows);
}
int or_assemble_system(const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                       const double* normals, const uint8_t* bc, double k, const double* dir,
                       int ng, int ng_near, cplx* A, cplx* b) {
  return assemble_system_n(nodes, N, elems, 6, E, normals, bc, k, dir, ng, ng_near, A, b);
}
/* Linear 3-node elements (Sec. 4's cross-check): the same equations with or_shape3. */
int or_assemble_raw_linear(const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                           const double* normals, double k, int ng, int ng_near, cplx* H, cplx* Gm,
                           cplx* alpha, cplx* beta) {
  return assemble_raw_n(nodes, N, elems, 3, E, normals, k, ng, ng_near, H, Gm, alpha, beta);
}
int or_assemble_system_linear(const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                              const double* normals, const uint8_t* bc, double k, const double* dir,
                              int ng, int ng_near, cplx* A, cplx* b) {
  return assemble_system_n(nodes, N, elems, 3, E, normals, bc, k, dir, ng, ng_near, A, b);
}

/* ------------------------------------------------------------------------------------------
 * Direct solution of the linear system (Sec. 4): textbook Doolittle LU with partial pivoting.
 * ------------------------------------------------------------------------------------------ */
int or_lu_factor(int64_t n, cplx* A, int64_t* piv) {
  for (int64_t k = 0; k < n; ++k) {
    int64_t p = k;
    double best = cabs(A[k * n + k]);
    for (int64_t r = k + 1; r < n; ++r) {
      double v = cabs(A[r * n + k]);
      if (v > best) { best = v; p = r; }
    }
    piv[k] = p;
    if (best == 0.0) return -4;
    if (p != k)
      for (int64_t c = 0; c < n; ++c) {
        cplx t = A[k * n + c]; A[k * n + c] = A[p * n + c]; A[p * n + c] = t;
      }
    cplx d = A[k * n + k];
#pragma omp parallel for schedule(static)
    for (int64_t r = k + 1; r < n; ++r) {
      cplx l = A[r * n + k] / d;
      A[r * n + k] = l;
      for (int64_t c = k + 1; c < n; ++c) A[r * n + c] -= l * A[k * n + c];
    }
  }
  return 0;
}

int or_lu_solve(int64_t n, const cplx* LU, const int64_t* piv, cplx* b) {
  for (int64_t k = 0; k < n; ++k)
    if (piv[k] != k) { cplx t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
  for (int64_t r = 0; r < n; ++r) { /* L y = P b, unit diagonal */
    cplx s = b[r];
    for (int64_t c = 0; c < r; ++c) s -= LU[r * n + c] * b[c];
    b[r] = s;
  }
  for (int64_t r = n - 1; r >= 0; --r) { /* U x = y */
    cplx s = b[r];
    for (int64_t c = r + 1; c < n; ++c) s -= LU[r * n + c] * b[c];
    b[r] = s / LU[r * n + r];
  }
  return 0;
}

int or_surface_fields(const double* nodes, int64_t N, const double* normals, const uint8_t* bc,
                      double k, const double* dir, const cplx* x, cplx* P, cplx* Pn) {
  for (int64_t j = 0; j < N; ++j) {
    cplx pinc = cexp(I * k * dot3(dir, nodes + 3 * j));
    if (bc[j] == 0) { P[j] = x[j]; Pn[j] = -(I * k * dot3(dir, normals + 3 * j)) * pinc; }
    else { P[j] = -pinc; Pn[j] = x[j]; }
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------
 * Closest surface point x0 of an observation point (Sec. 3, after Eq. BRIEFdmn).
 * ------------------------------------------------------------------------------------------ */
/* Constant second derivatives of the six shape functions: (xi xi, xi eta, eta eta). */
static const double D2N[6][3] = {{4, 4, 4}, {4, 0, 0}, {0, 0, 4}, {-8, -4, 0}, {0, 4, 0}, {0, -4, -8}};

static void clamp_tri(double* xi, double* eta) {
  if (*xi < 0) *xi = 0;
  if (*eta < 0) *eta = 0;
  if (*xi + *eta > 1.0) {
    double t = 0.5 * (*xi + *eta - 1.0);
    *xi -= t;
    *eta -= t;
    if (*xi < 0) { *xi = 0; *eta = 1; }
    if (*eta < 0) { *eta = 0; *xi = 1; }
  }
}

static double dist2_at(const double* nodes, const int32_t* el, int np, double xi, double eta, const double* p) {
  double x[3], nu[3], J, Nv[6];
  elem_point(nodes, el, np, xi, eta, x, nu, &J, Nv);
  double d[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
  return dot3(d, d);
}

/* Damped Newton minimisation of |x(xi,eta) - p|^2 over the reference triangle (a linear element,
 * np = 3, has no second derivatives). */
static double project_elem(const double* nodes, const int32_t* el, int np, const double* p, double* pxi,
                           double* peta) {
  double xi = *pxi, eta = *peta;
  double f = dist2_at(nodes, el, np, xi, eta, p);
  for (int it = 0; it < 100; ++it) {
    double Nv[6], dx[6], de[6];
    shape_n(np, xi, eta, Nv, dx, de);
    double x[3] = {0, 0, 0}, t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0}, xx[3] = {0, 0, 0},
           xe[3] = {0, 0, 0}, ee[3] = {0, 0, 0};
    for (int a = 0; a < np; ++a) {
      const double* X = nodes + 3 * (int64_t)el[a];
      for (int d = 0; d < 3; ++d) {
        x[d] += Nv[a] * X[d];
        t1[d] += dx[a] * X[d];
        t2[d] += de[a] * X[d];
        if (np == 6) {
          xx[d] += D2N[a][0] * X[d];
          xe[d] += D2N[a][1] * X[d];
          ee[d] += D2N[a][2] * X[d];
        }
      }
    }
    double r[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
    double g1 = dot3(r, t1), g2 = dot3(r, t2);
    double a11 = dot3(t1, t1) + dot3(r, xx), a12 = dot3(t1, t2) + dot3(r, xe),
           a22 = dot3(t2, t2) + dot3(r, ee);
    double det = a11 * a22 - a12 * a12;
    if (!(a11 > 0 && det > 0)) { /* not convex here: Gauss-Newton matrix instead */
      a11 = dot3(t1, t1); a12 = dot3(t1, t2); a22 = dot3(t2, t2);
      det = a11 * a22 - a12 * a12;
    }
    double s1 = -(a22 * g1 - a12 * g2) / det, s2 = -(a11 * g2 - a12 * g1) / det;
    double lam = 1.0, nxi = xi, neta = eta, nf = f;
    int accepted = 0;
    if (fabs(s1) + fabs(s2) < 1e-6) { /* inside the quadratic region: plain Newton step, since
                                         changes of |x - p|^2 there are below its rounding */
      nxi = xi + s1;
      neta = eta + s2;
      clamp_tri(&nxi, &neta);
      nf = dist2_at(nodes, el, np, nxi, neta, p);
      accepted = 1;
    }
    for (int h = 0; h < 40 && !accepted; ++h) {
      nxi = xi + lam * s1;
      neta = eta + lam * s2;
      clamp_tri(&nxi, &neta);
      nf = dist2_at(nodes, el, np, nxi, neta, p);
      if (nf <= f) { accepted = 1; break; }
      lam *= 0.5;
    }
    if (!accepted) break;
    double moved = fabs(nxi - xi) + fabs(neta - eta);
    xi = nxi; eta = neta; f = nf;
    if (moved < 1e-15) break;
  }
  *pxi = xi;
  *peta = eta;
  return f;
}

static int foot_points_n(const double* nodes, int64_t N, const int32_t* elems, int np, int64_t E,
                         const double* xp, int64_t M, int32_t* foot_elem, double* foot_xi,
                         double* foot_eta) {
  if (N < 1 || E < 1 || M < 0) return -1;
#pragma omp parallel for schedule(static)
  for (int64_t m = 0; m < M; ++m) {
    const double* p = xp + 3 * m;
    int64_t best_node = 0;
    double bd = INFINITY;
    for (int64_t j = 0; j < N; ++j) {
      double d[3] = {nodes[3 * j] - p[0], nodes[3 * j + 1] - p[1], nodes[3 * j + 2] - p[2]};
      double d2 = dot3(d, d);
      if (d2 < bd) { bd = d2; best_node = j; }
    }
    double best = INFINITY;
    int32_t be = -1;
    double bxi = 0, beta_ = 0;
    for (int64_t e = 0; e < E; ++e) {
      const int32_t* el = elems + (int64_t)np * e;
      int own = -1;
      for (int a = 0; a < np; ++a)
        if (el[a] == best_node) own = a;
      if (own < 0) continue;
      double xi = REF_NODE[own][0], eta = REF_NODE[own][1];
      double f = project_elem(nodes, el, np, p, &xi, &eta);
      if (f < best) { best = f; be = (int32_t)e; bxi = xi; beta_ = eta; }
    }
    foot_elem[m] = be;
    foot_xi[m] = bxi;
    foot_eta[m] = beta_;
  }
  return 0;
}

int or_foot_points(const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                   const double* xp, int64_t M, int32_t* foot_elem, double* foot_xi,
                   double* foot_eta) {
  return foot_points_n(nodes, N, elems, 6, E, xp, M, foot_elem, foot_xi, foot_eta);
}
int or_foot_points_linear(const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                          const double* xp, int64_t M, int32_t* foot_elem, double* foot_xi,
                          double* foot_eta) {
  return foot_points_n(nodes, N, elems, 3, E, xp, M, foot_elem, foot_xi, foot_eta);
}

/* ------------------------------------------------------------------------------------------
 * Field at observation points, Eq. BRIEFdmn (S-only form: the S_inf integrals of g and f about
 * x0 and x_p cancel against the 4 pi [P0 g(x_p) + P0' f(x_p)] term, leaving 4 pi P0).
 * ------------------------------------------------------------------------------------------ */
static int field_n(const double* nodes, int64_t N, const int32_t* elems, int np, int64_t E, double k, int ng,
                   const cplx* P, const cplx* Pn, const double* xp, int64_t M, const int32_t* foot_elem,
                   const double* foot_xi, const double* foot_eta, cplx* T) {
  if (N < 1 || E < 1 || !(k >= 0.0) || ng < 1 || ng > 16) return -1;
  double sxi[256], seta[256], sw[256];
  int nq = or_rule_std(ng, sxi, seta, sw);
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t m = 0; m < M; ++m) {
    const double* p = xp + 3 * m;
    const int32_t* el0 = elems + (int64_t)np * foot_elem[m];
    double x0[3], nu0[3], J0, N0[6];
    elem_point(nodes, el0, np, foot_xi[m], foot_eta[m], x0, nu0, &J0, N0);
    cplx P0 = 0.0, Pn0 = 0.0; /* interpolation at the foot point (quadratic, or linear for np = 3) */
    for (int a = 0; a < np; ++a) { P0 += N0[a] * P[el0[a]]; Pn0 += N0[a] * Pn[el0[a]]; }
    cplx sum = 0.0;
    for (int64_t e = 0; e < E; ++e) {
      const int32_t* el = elems + (int64_t)np * e;
      for (int q = 0; q < nq; ++q) {
        double x[3], nu[3], J, Nv[6];
        elem_point(nodes, el, np, sxi[q], seta[q], x, nu, &J, Nv);
        cplx Pq = 0.0, Pnq = 0.0;
        for (int a = 0; a < np; ++a) { Pq += Nv[a] * P[el[a]]; Pnq += Nv[a] * Pn[el[a]]; }
        double rp[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
        double r0[3] = {x[0] - x0[0], x[1] - x0[1], x[2] - x0[2]};
        double Rp = sqrt(dot3(rp, rp)), R0 = sqrt(dot3(r0, r0));
        cplx ep = cexp(I * k * Rp), e0 = cexp(I * k * R0);
        cplx Gp = ep / Rp, G0 = e0 / R0;
        cplx dGp = ep * (I * k * Rp - 1.0) * dot3(rp, nu) / (Rp * Rp * Rp);
        cplx dG0 = e0 * (I * k * R0 - 1.0) * dot3(r0, nu) / (R0 * R0 * R0);
        double s = k * dot3(nu0, r0);
        double g = cos(s), f = (k == 0.0) ? dot3(nu0, r0) : sin(s) / k; /* k = 0: the limit nu0.r0 */
        double dg = -k * sin(s) * dot3(nu0, nu), df = cos(s) * dot3(nu0, nu);
        cplx Pt = Pq - P0 * g - Pn0 * f;
        cplx dPt = Pnq - P0 * dg - Pn0 * df;
        sum += sw[q] * J * (Pt * (dGp - dG0) - (Gp - G0) * dPt);
      }
    }
    T[m] = P0 + sum / (4.0 * PI);
  }
  return 0;
}

int or_field(const double* nodes, int64_t N, const int32_t* elems, int64_t E, double k, int ng,
             const cplx* P, const cplx* Pn, const double* xp, int64_t M, const int32_t* foot_elem,
             const double* foot_xi, const double* foot_eta, cplx* T) {
  return field_n(nodes, N, elems, 6, E, k, ng, P, Pn, xp, M, foot_elem, foot_xi, foot_eta, T);
}
int or_field_linear(const double* nodes, int64_t N, const int32_t* elems, int64_t E, double k, int ng,
                    const cplx* P, const cplx* Pn, const double* xp, int64_t M, const int32_t* foot_elem,
                    const double* foot_xi, const double* foot_eta, cplx* T) {
  return field_n(nodes, N, elems, 3, E, k, ng, P, Pn, xp, M, foot_elem, foot_xi, foot_eta, T);
}

/* ------------------------------------------------------------------------------------------
 * Fourier transforms with the sign convention of Eq. inverseFourier (exp(-i omega t)).
 * ------------------------------------------------------------------------------------------ */
int or_dft(int64_t Nt, const double* s, cplx* S) {
  if (Nt < 1) return -1;
#pragma omp parallel for schedule(static)
  for (int64_t m = 0; m < Nt; ++m) {
    cplx acc = 0.0;
    for (int64_t n = 0; n < Nt; ++n) {
      int64_t ph = (m * n) % Nt; /* exact phase index */
      acc += s[n] * cexp(I * 2.0 * PI * (double)ph / (double)Nt);
    }
    S[m] = acc;
  }
  return 0;
}

int or_synthesize(int64_t Nk, int64_t M, const cplx* T, const int64_t* midx, int64_t P,
                  int64_t Nt, const cplx* S, double* p) {
  if (Nt < 2 || (Nt & 1) || Nk < 0 || M < 0 || P < 0) return -1;
  for (int64_t r = 0; r < Nk; ++r)
    if (midx[r] < 0 || midx[r] > Nt / 2) return -1;
#pragma omp parallel for schedule(static)
  for (int64_t pm = 0; pm < P * M; ++pm) {
    int64_t ip = pm / M, x = pm % M;
    for (int64_t n = 0; n < Nt; ++n) {
      double acc = 0.0;
      for (int64_t r = 0; r < Nk; ++r) {
        int64_t m = midx[r];
        double wgt = (m == 0 || 2 * m == Nt) ? 1.0 : 2.0;
        int64_t ph = (m * n) % Nt;
        cplx term = S[ip * Nt + m] * T[r * M + x] * cexp(-I * 2.0 * PI * (double)ph / (double)Nt);
        acc += wgt * creal(term);
      }
      p[pm * Nt + n] = acc / (double)Nt;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------
 * Dominant frequencies (Sec. 4, Table I): the K indices m (0 <= m <= Nt/2) with the largest
 * amplitude max_p |S[p][m]| of the incident spectra, ties to the lower m, returned ascending.
 * Plain repeated selection of the largest remaining amplitude.
 * ------------------------------------------------------------------------------------------ */
int or_top_frequencies(int64_t P, int64_t Nt, const cplx* S, int64_t K, int64_t* midx) {
  const int64_t nm = Nt / 2 + 1;
  if (P < 1 || Nt < 2 || K < 0 || K > nm) return -1;
  double* amp = (double*)malloc(sizeof(double) * nm);
  char* taken = (char*)calloc(nm, 1);
  if (!amp || !taken) { free(amp); free(taken); return -3; }
  for (int64_t m = 0; m < nm; ++m) {
    amp[m] = 0.0;
    for (int64_t p = 0; p < P; ++p) {
      double a = cabs(S[p * Nt + m]);
      if (a > amp[m]) amp[m] = a;
    }
  }
  for (int64_t r = 0; r < K; ++r) {
    int64_t best = -1;
    for (int64_t m = 0; m < nm; ++m)
      if (!taken[m] && (best < 0 || amp[m] > amp[best])) best = m;
    taken[best] = 1;
  }
  int64_t c = 0;
  for (int64_t m = 0; m < nm; ++m)
    if (taken[m]) midx[c++] = m;
  free(amp);
  free(taken);
  return 0;
}
