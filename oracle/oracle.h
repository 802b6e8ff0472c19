/* oracle.h -- plain, slow, obviously-correct CPU FP64 restatement of the non-singular boundary
 * integral method of Klaseboer, Sepehrirahnama & Chan (arXiv 1706.07919).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or includes this
 * code; only the tests, the smoke check and the benchmark's CPU-baseline leg use it.  It shares
 * no code with the CUDA path (no headers, helpers, tables or generated constants).
 *
 * Conventions (units a = c = 1):
 *   complex numbers are C99 `double _Complex` (interleaved re, im);
 *   matrices are row-major;
 *   element node order v0 v1 v2 m01 m12 m20, reference triangle (0,0) (1,0) (0,1);
 *   node normals nu point out of the scatterer into the fluid;
 *   bc[j] = 0 sound-hard (dp/dn = 0), 1 sound-soft (p = 0);
 *   time dependence exp(-i omega t) (Eq. inverseFourier), G = exp(ikR)/R (Eq. Green_func).
 * All functions return 0 on success and a negative value on invalid input.
 */
#ifndef BIE_ORACLE_H
#define BIE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Gauss-Legendre nodes/weights on [0,1] by Newton iteration on P_n. */
int or_gauss_legendre01(int n, double* x, double* w);

/* Quadratic 6-node shape functions and their parametric derivatives at (xi, eta) (Sec. 3). */
void or_shape6(double xi, double eta, double* N, double* dNxi, double* dNeta);

/* Linear 3-node shape functions (the barycentric coordinates) and their derivatives (Sec. 4: the
 * cross-check with linear elements and linear interpolation). */
void or_shape3(double xi, double eta, double* N, double* dNxi, double* dNeta);

/* Standard rule: n*n collapsed (Duffy) Gauss-Legendre points on the reference triangle,
 * collapsed at vertex 0.  Returns the point count. */
int or_rule_std(int n, double* xi, double* eta, double* w);

/* Near rule for an element whose local node `a` is the collocation node: the triangle is
 * split at that node into 1 (vertex) or 2 (mid-edge) sub-triangles, each Duffy-collapsed
 * onto the node, n*n points each.  Returns the point count (n*n or 2*n*n). */
int or_rule_near(int n, int a, double* xi, double* eta, double* w);

/* Raw discretised integrals of Eq. BRIEF at every node x_i (Sec. 3, App. A):
 *   H[i][j]  = sum_{e,q} w J N_a dG(x_i,x_q)/dnu_q       (j = node a of e)
 *   Gm[i][j] = sum_{e,q} w J N_a G(x_i,x_q)
 *   alpha[i] = sum_{e,q} w J [g_i dG/dnu - dg_i/dnu G],  beta[i] = same with f_i
 * with g_i = cos(k nu_i.(x-x_i)), f_i = sin(k nu_i.(x-x_i))/k (Eqs. f_function, g_function).
 * k >= 0: at k = 0 (the zero-frequency term of Eq. inverseFourier, the Laplace limit) the same
 * formulas hold with f_i replaced by its limit nu_i.(x-x_i); G = 1/R, g = 1, dg = 0.
 * Elements that contain node i use the near rule (ng_near), the others the standard rule (ng). */
int or_assemble_raw(const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                    const double* normals, double k, int ng, int ng_near,
                    double _Complex* H, double _Complex* Gm, double _Complex* alpha,
                    double _Complex* beta);

/* Linear system of the scattered field (Eq. BRIEF with the S_inf term of App. B; BCs of Sec. 4):
 *   row i:  sum_j [H_ij - (4 pi + alpha_i) d_ij] P_j - sum_j [Gm_ij + beta_i d_ij] P'_j = 0,
 * unknown P_j at hard nodes, P'_j at soft nodes; known P'_j = -dP_inc/dnu (hard),
 * P_j = -P_inc (soft), P_inc = exp(i k d.x).  A is N x N, b has N entries. */
int or_assemble_system(const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                       const double* normals, const uint8_t* bc, double k, const double* dir,
                       int ng, int ng_near, double _Complex* A, double _Complex* b);

/* The rows rows[0..nrows) of that system (the same arithmetic, row by row): A_rows [nrows][N],
 * b_rows [nrows]; for checks at sizes where the whole system does not fit. */
int or_assemble_rows(const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                     const double* normals, const uint8_t* bc, double k, const double* dir, int ng,
                     int ng_near, const int64_t* rows, int64_t nrows, double _Complex* A_rows,
                     double _Complex* b_rows);

/* The same three functions for linear 3-node elements (elems [E][3], vertices counter-clockwise
 * seen from the fluid; flat geometry, linear interpolation of P and dP/dnu, or_shape3), with
 * collocation at the vertices; the near rule of a vertex as for quadratic elements. */
int or_assemble_raw_linear(const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                           const double* normals, double k, int ng, int ng_near,
                           double _Complex* H, double _Complex* Gm, double _Complex* alpha,
                           double _Complex* beta);
int or_assemble_system_linear(const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                              const double* normals, const uint8_t* bc, double k, const double* dir,
                              int ng, int ng_near, double _Complex* A, double _Complex* b);

/* Dense complex LU with partial pivoting (largest modulus, ties to the lowest row), in place;
 * piv[k] = row swapped with row k.  Returns 0, or -4 on an exactly zero pivot. */
int or_lu_factor(int64_t n, double _Complex* A, int64_t* piv);
/* Solve with the factor from or_lu_factor; b is overwritten by x. */
int or_lu_solve(int64_t n, const double _Complex* LU, const int64_t* piv, double _Complex* b);

/* Surface scattered field (P, dP/dnu) at every node from the solution x and the BCs. */
int or_surface_fields(const double* nodes, int64_t N, const double* normals, const uint8_t* bc,
                      double k, const double* dir, const double _Complex* x,
                      double _Complex* P, double _Complex* Pn);

/* Closest-point foot x0 for each observation point (Sec. 3 after Eq. BRIEFdmn): nearest node
 * (lowest index on ties), then a damped Newton projection onto each element containing that
 * node, the smallest distance winning (lowest element index on ties). */
int or_foot_points(const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                   const double* xp, int64_t M, int32_t* foot_elem, double* foot_xi,
                   double* foot_eta);

/* Scattered field T(x_p) per unit incident amplitude from the surface solution, by the
 * boundary-regularised representation Eq. BRIEFdmn with its S_inf parts evaluated analytically
 * (App. B reasoning): 4 pi P(x_p) = 4 pi P0 + int_S Pt (dG_p - dG_0) - (G_p - G_0) dPt dS,
 * Pt = P - P0 g - P0' f about the foot point x0; standard rule on every element.  k >= 0, with
 * f -> nu0.(x - x0) at k = 0 as in or_assemble_raw. */
int or_field(const double* nodes, int64_t N, const int32_t* elems, int64_t E, double k, int ng,
             const double _Complex* P, const double _Complex* Pn, const double* xp, int64_t M,
             const int32_t* foot_elem, const double* foot_xi, const double* foot_eta,
             double _Complex* T);

/* or_foot_points and or_field for linear 3-node elements. */
int or_foot_points_linear(const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                          const double* xp, int64_t M, int32_t* foot_elem, double* foot_xi,
                          double* foot_eta);
int or_field_linear(const double* nodes, int64_t N, const int32_t* elems, int64_t E, double k, int ng,
                    const double _Complex* P, const double _Complex* Pn, const double* xp, int64_t M,
                    const int32_t* foot_elem, const double* foot_xi, const double* foot_eta,
                    double _Complex* T);

/* Naive DFT of a sampled pulse with the sign of Eq. inverseFourier:
 * S_m = sum_n s_n exp(+2 pi i m n / Nt), m = 0..Nt-1. */
int or_dft(int64_t Nt, const double* s, double _Complex* S);

/* Naive inverse transform (Sec. 3 last paragraph, Sec. 4) of the spectra weighted by each pulse:
 *   p[P][M][n] = (1/Nt) sum_rows w_m Re( S[p][m] T[row][x] exp(-2 pi i m n / Nt) )
 * row r carries frequency index m = midx[r] (0 <= m <= Nt/2), w_m = 1 for m = 0 or Nt/2,
 * else 2 (Hermitian symmetry of a real signal); absent frequencies count as zero. */
int or_synthesize(int64_t Nk, int64_t M, const double _Complex* T, const int64_t* midx,
                  int64_t P, int64_t Nt, const double _Complex* S, double* p);

/* Dominant frequencies (Sec. 4, Table I): the K indices m in [0, Nt/2] of largest
 * max_p |S[p][m]| (S [P][Nt], full spectra as or_dft writes them), ties to the lower m,
 * written ascending to midx [K]. */
int or_top_frequencies(int64_t P, int64_t Nt, const double _Complex* S, int64_t K, int64_t* midx);

/* ---- learned warm start of the frequency sweep (not part of the paper's method) -------------
 * Feature map, network, loss and optimiser step are defined in full at the top of mlp.c; the
 * parameter vector is W1 (256x64) | b1 | W2 (256x256) | b2 | W3 (256x256) | b3 | W4 (2x256) | b4. */
int64_t or_mlp_param_count(void);
/* phi[nk][N][64] for nodes x[N][3] with normals nu[N][3] at wavenumbers kv[nk]. */
int or_mlp_features(const double* x, const double* nu, int64_t N, const double* kv, int64_t nk,
                    const double* dir, const double* centre, double scale, double kmax, double* phi);
/* Y[B][2] = network(X[B][64]). */
int or_mlp_forward(const double* theta, const double* X, int64_t B, double* Y);
/* loss = (1/B) sum |Y - T|^2 and its gradient with respect to theta (analytic backward). */
int or_mlp_loss_grad(const double* theta, const double* X, const double* T, int64_t B, double* loss,
                     double* grad);
int or_mlp_loss(const double* theta, const double* X, const double* T, int64_t B, double* loss);
/* One Adam step (step counter t >= 1) on P parameters, in place on theta, m, v. */
int or_adam_step(int64_t P, double* theta, const double* grad, double* m, double* v, int64_t t, double lr,
                 double beta1, double beta2, double eps);

/* Number of OpenMP threads the oracle uses. */
int or_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
