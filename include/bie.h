/* bie.h -- C ABI of the GB300 library for the space-time boundary-regularised (non-singular)
 * boundary integral method of Klaseboer, Sepehrirahnama & Chan, "Space-time domain solutions of
 * the wave equation by a non-singular boundary integral method and Fourier transform"
 * (arXiv 1706.07919).
 *
 * Problem statement (Sec. 4): scatterers bounded by surfaces S, meshed with quadratic 6-node
 * triangles (Sec. 3), sound-hard or sound-soft, are hit by a plane-wave pulse train.  For every
 * wavenumber k the library solves the frequency-domain boundary integral equation Eq. (BRIEF)
 * -- kernels regularised by the functions g and f of App. A, the surface at infinity evaluated
 * analytically (App. B) -- for the scattered surface pressure P or dP/dn, evaluates the scattered
 * field at observation points by Eq. (BRIEFdmn), and synthesises p_scat(x, t) for any number of
 * incident pulses by the inverse discrete Fourier transform (Eq. inverseFourier, Sec. 3 end).
 *
 * Conventions, used by every entry point:
 *   units a = c = 1; time dependence exp(-i omega t); G(x, y) = exp(ik|x-y|)/|x-y|;
 *   complex values are interleaved (re, im) doubles ("c128") unless stated;
 *   node normals point out of the scatterer into the fluid;
 *   element node order v0 v1 v2 m01 m12 m20, counter-clockwise seen from the fluid;
 *   bc[j] = 0: sound-hard node (dp/dn = 0), 1: sound-soft node (p = 0);
 *   the incident field per unit amplitude at wavenumber k is exp(i k d.x) (unit vector d).
 * Memory: pointers documented "host" are read (or written) during the call only; pointers
 * documented "device" must be device memory of the context's GPU, are used on the context's
 * stream, and stay owned by the caller.  Calls are stream-ordered: they return once their work
 * is enqueued (except where stated), and device outputs are valid after the stream completes.
 * Errors: every function returns BIE_OK (0) or a negative BIE_ERR_* code and then leaves a
 * message in bie_last_error() (thread-local).  No C++ exception crosses this interface and the
 * library never traps the device.
 */
#ifndef BIE_H
#define BIE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BIE_OK 0
#define BIE_ERR_INVALID_ARG (-1)
#define BIE_ERR_CUDA (-2)
#define BIE_ERR_OOM (-3)
#define BIE_ERR_SINGULAR (-4)
#define BIE_ERR_NOT_CONVERGED (-5)
#define BIE_ERR_TIMEOUT (-6)
#define BIE_ERR_STATE (-7)

/* Precision modes of bie_solve_frequencies. */
#define BIE_MODE_FP64 0   /* FP64 assembly, FP64 LU with partial pivoting, FP64 solve */
#define BIE_MODE_MIXED 1  /* FP32 assembly (float-float distance/phase), TF32 tcgen05 LU,
                             iterative refinement with float-float residuals */
#define BIE_MODE_LEARNED 2 /* every "learned.stride"-th wavenumber ("anchor") solved as
                             BIE_MODE_MIXED, keeping its low-precision factor; a network trained on
                             the anchors' solutions predicts the others, which are solved by
                             flexible GMRES from that guess, preconditioned by the nearest anchor's
                             factor (see bie_set_option); not part of the paper's method */

/* Parameter count of the learned warm start's network (see bie_mlp_set_params). */
#define BIE_MLP_PARAMS 148738

/* Report flags (bie_report.flags). */
#define BIE_FLAG_NOT_CONVERGED 1u   /* refinement stopped at its iteration cap */
#define BIE_FLAG_FALLBACK_FP64 2u   /* the frequency was re-solved by the FP64 path (its report then
                                       describes that solve: path BIE_MODE_FP64, NOT_CONVERGED
                                       cleared) */
#define BIE_FLAG_ZERO_PIVOT 4u      /* an exactly zero pivot was met */
#define BIE_FLAG_ILL_CONDITIONED 8u /* the FP32 assembly's rounding, pushed through the solve, was
                                       estimated above "mixed.fallback_err_est" (a wavenumber
                                       near an interior resonance) */
#define BIE_FLAG_FP64_ASSEMBLY 16u  /* re-assembled in FP64 and refined against that system with
                                       the low-precision factor (after ILL_CONDITIONED or a stalled
                                       refinement); if that also stalls, FP32_REFACTOR or, when
                                       the re-factorisation stalls too, FALLBACK_FP64 is added */
#define BIE_FLAG_FP32_REFACTOR 32u  /* the TF32 factor's refinement against the FP64 re-assembly
                                       stalled (or that factor met a zero pivot); the FP64 system
                                       was factored again in FP32 on the CUDA cores and refined with
                                       that factor (bie_solve_frequencies; FP64_ASSEMBLY set too) */

typedef struct bie_ctx bie_ctx;

/* Per-frequency outcome of bie_solve_frequencies (host array, valid when that call returns). */
typedef struct {
  int32_t iters;        /* refinement iterations (0 for the FP64 path); Arnoldi steps for
                           wavenumbers solved by GMRES in BIE_MODE_LEARNED */
  int32_t path;         /* BIE_MODE_* that produced the result */
  uint32_t flags;       /* BIE_FLAG_* bits */
  int32_t reserved;
  double backward_err;  /* ||b - A x|| / (||A||_inf ||x|| + ||b||), infinity norms, of the
                           refinement or Krylov solve; 0 for the FP64 path (a direct solve
                           with partial pivoting, not measured) */
  double err_est;       /* mixed path: estimated relative L2 error of x caused by the FP32
                           assembly (a seeded FP32-sized perturbation of A solved with the LU) */
} bie_report;

/* Summary of the last BIE_MODE_LEARNED call (bie_get_learned_info()). */
typedef struct {
  int32_t anchors;         /* wavenumbers solved directly */
  int32_t krylov;          /* wavenumbers solved by GMRES */
  int32_t krylov_fallback; /* of those, re-solved directly (GMRES did not converge) */
  int32_t epochs;          /* training epochs run */
  float first_loss;        /* mean minibatch loss of the first and last epoch (targets scaled to */
  float last_loss;         /*   unit mean square) */
  double train_ms;         /* wall time of the training */
  double x0_rel_err;       /* mean over GMRES-solved wavenumbers of ||x0 - x|| / ||x|| */
  double mean_iters;       /* mean Arnoldi steps per GMRES-solved wavenumber */
  double max_iters;        /* largest Arnoldi step count of a GMRES-solved wavenumber */
  double anchors_ms;       /* device time of the anchors' direct solves */
  double assembly_ms;      /* device time of the GMRES-solved wavenumbers' assembly */
  double predict_ms;       /* device time of the initial guesses */
  double gmres_ms;         /* device time of the GMRES solves */
  double estimate_ms;      /* device time of the sensitivity estimates */
  double redo_ms;          /* wall time of the direct re-solves of handed-back wavenumbers */
} bie_learned_info;

/* Result of bie_autotune. */
typedef struct {
  int32_t n_bucket;    /* N rounded up to a multiple of 64: the cache key */
  int32_t batch;       /* wavenumbers per batch chosen ("mixed.batch") */
  int32_t tcgen05;     /* trailing-update kernel chosen ("mixed.tcgen05") */
  int32_t from_cache;  /* 1: read from the cache file, 0: measured now */
  double us_per_k;     /* measured time per wavenumber of the chosen setting */
  int32_t lu_block;    /* columns over which the deferred update runs ("mixed.lu_block") */
  int32_t lu_panel;    /* panel width of the deferred version ("mixed.lu_panel") */
  int32_t lu_tile;     /* real columns of the update tile ("mixed.lu_tile") */
} bie_tune_result;

/* Device time of the phases of the last BIE_MODE_MIXED call (bie_get_phase_times), recorded
 * with CUDA events on the context's stream when the option "mixed.phase_timing" is 1. */
typedef struct {
  double assembly_ms;    /* FP32 assembly of every batch (with the copy of A into the factor) */
  double factor_ms;      /* blocked LU of every batch: panels and tensor-core trailing updates */
  double refine_ms;      /* diagonal-block inverses, refinement and sensitivity estimates */
  double reassembly_ms;  /* re-assembly and refinement of flagged wavenumbers */
  int32_t batches;       /* batches timed */
  int32_t systems;       /* wavenumbers factored */
  int32_t reassembled;   /* wavenumbers re-assembled */
  int32_t reserved;
} bie_phase_times;

/* Rates of the pipes that bound the library's kernels, measured by bie_measure_peaks. */
typedef struct {
  double ffma_tflops;  /* FP32 fused multiply-add (2 flops each), all SMs */
  double dfma_tflops;  /* FP64 fused multiply-add */
  double tf32_tflops;  /* tcgen05.mma kind::tf32, M = 128, N = 256, dense, 0 if not sm_100-family */
  double bf16_tflops;  /* tcgen05.mma kind::f16 with BF16 operands, same shape */
  int32_t sm_count;
  int32_t reserved;
} bie_peaks;

/* Statistics of bie_sched_run. */
typedef struct {
  int32_t jobs, workers;
  double wall_ms;  /* wall time of the whole run */
  double busy_ms;  /* sum over workers of the time spent inside jobs */
} bie_sched_stats;

typedef struct bie_sched bie_sched;

/* Message of the last failed call on this thread ("" if none). */
const char* bie_last_error(void);

/* Library version string. */
const char* bie_version(void);

/* Number of CUDA kernels this library has enqueued since it was loaded (all contexts and
 * threads); a diagnostic for counting launches in a region of interest. */
uint64_t bie_kernel_launches(void);

/* Creates a context on CUDA device `cuda_device` that enqueues on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  *out receives the handle.  The context owns
 * its device scratch (allocated on demand, released by bie_destroy).  Errors: INVALID_ARG for a
 * bad device index or NULL out, CUDA if the device cannot be used. */
int bie_create(bie_ctx** out, int cuda_device, void* cuda_stream);

/* Synchronises the context's stream and frees everything it owns. NULL is accepted. */
int bie_destroy(bie_ctx* ctx);

/* Quadrature (Sec. 3: ordinary Gauss quadrature on regular integrands): ng x ng collapsed Gauss-Legendre
 * points per element (default 4), and ng_near x ng_near per sub-triangle for elements that
 * contain the collocation node (default 6), which are split at that node and collapsed onto it.
 * Must precede bie_set_geometry to take effect on it.  Errors: INVALID_ARG unless
 * 1 <= ng <= 8 and 1 <= ng_near <= 12. */
int bie_set_quadrature(bie_ctx* ctx, int ng, int ng_near);

/* Surface mesh of all scatterers (Sec. 3 and 4).
 *   nodes   host f64 [N][3]  node positions
 *   elems   host i32 [E][6]  element nodes, order above, 0 <= index < N
 *   normals host f64 [N][3]  unit node normals into the fluid (used for f, g of App. A at
 *                            collocation nodes and for dP/dn); NULL: the normalised mean of the
 *                            adjacent elements' normals at the node
 *   bc      host u8  [N]     0 hard, 1 soft
 * Copied to the device; the geometry precompute (quadrature points, element colouring, near
 * lists) runs once here.  Errors: INVALID_ARG for N < 3, E < 1, an index out of range, a
 * non-finite coordinate, a zero-area element or a zero normal; CUDA/OOM on device failures. */
int bie_set_geometry(bie_ctx* ctx, const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                     const double* normals, const uint8_t* bc);

/* Surface mesh of linear 3-node elements (Sec. 4: the paper's cross-check of its quadratic-element
 * results with 774 flat linear elements and 389 nodes, linear interpolation on each element):
 *   nodes host f64 [N][3], elems host i32 [E][3] (vertices counter-clockwise seen from the fluid),
 *   normals host f64 [N][3] or NULL (as bie_set_geometry), bc host u8 [N]; every element must
 *   carry one boundary condition on its three vertices.
 * The library forms the flat quadratic image of the mesh (one mid-edge node per edge at its
 * midpoint; on it, quadratic interpolation of the vertex values' linear interpolant is exact),
 * assembles that system with its own kernels and reduces it to the vertex unknowns (rows of the
 * vertices, each mid-edge column shared half and half by its two vertices) -- exactly the
 * linear-element system.  Afterwards bie_assemble returns the [N][N] linear system,
 * bie_solve_frequencies (BIE_MODE_FP64 only) writes surf [Nk][2][N] at the vertices, and
 * bie_eval_field takes that surf (interpolated linearly onto the image for Eq. BRIEFdmn).
 * Errors: as bie_set_geometry; INVALID_ARG for an element with two conditions or an image of more
 * than 25 600 nodes (N + number of edges). */
int bie_set_geometry_linear(bie_ctx* ctx, const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                            const double* normals, const uint8_t* bc);

/* Direction d (host f64[3], normalised here) of the incident plane wave exp(i k d.x) (Sec. 4).
 * Default (0, 0, 1).  Errors: INVALID_ARG for a zero or non-finite vector. */
int bie_set_incident_plane_wave(bie_ctx* ctx, const double* dir);

/* Tuning options of the mixed-precision path (names are case-sensitive):
 *   "mixed.tcgen05"        trailing LU update: 3 (default) persistent TMA-fed tcgen05 kernel
 *                          (TF32 operands, FP32 accumulation in TMEM) with the update of the
 *                          trailing matrix deferred over blocks of "mixed.lu_block" columns,
 *                          2 the same kernel after every 64-column panel, 1 the
 *                          register-staged tcgen05 kernel, 0 FP32 on the CUDA cores.
 *   "mixed.lu_block"       columns of the deferred update of version 3: 128, 256, 512, or 0
 *                          (default): 512 from N = 8192 on, else 256
 *   "mixed.lu_coop"        1 (default): the panels of few tall matrices (at most half as many
 *                          matrices as SMs, more than 1536 rows) are factored by several CTAs per
 *                          matrix in one cooperative launch; 0: one CTA per matrix always
 *   "mixed.lu_panel"       panel width of version 3: 64 (default) or 32 (more, narrower panels:
 *                          shorter pivot chains per leaf, narrower K = 32 updates inside a block)
 *   "mixed.lu_tile"        tile of the tensor-core update (versions 2, 3): 128 rows x 256 real
 *                          columns (default; MMA N = 256) or 128 x 128 (MMA N = 128)
 *   "mixed.batch"          wavenumbers factored per batch (>= 1, default 256; at most as many as
 *                          half the free device memory holds)
 *   "refine.tol"           backward-error target of iterative refinement (default 1e-11)
 *   "refine.it_max"        refinement corrections per wavenumber (0..64, default 10)
 *   "mixed.fallback_err_est" FP64 re-assembly when the estimated error exceeds it (default 3e-7)
 *   "mixed.refine64_it_max" corrections against the FP64 re-assembly (0..64, default 30); if they
 *                          do not reach a backward error of 1e-13, the FP64 system is factored
 *                          again in FP32 and refined with that factor (up to 30 corrections), and
 *                          if that also stalls the full FP64 path solves it
 *   "mixed.refactor32"     1 (default): take the FP32 re-factorisation step above; 0: go from the
 *                          stalled refinement straight to the full FP64 path
 *   "field.accurate_phase" 1: float-float phases in the mixed field evaluation (default),
 *                          0: FP32 phases with hardware sine/cosine
 *   "field.variant"        mixed field kernel: 2 (default) groups of 16 wavenumbers, 128 points per
 *                          CTA, tiles of 32 quadrature points, FP32 run sums; 1 the same with 64
 *                          points per CTA and 64-point tiles; 0 groups of 8, 128 points,
 *                          compensated sums per term
 *   "mixed.asm_kb"         FP32 bulk assembly on meshes whose elements carry one boundary
 *                          condition each: 2 (default) wavenumbers per thread, 1, or 0 (the general
 *                          kernel, one wavenumber per thread, both nodal sums per element)
 *   "asm.windows"          1 (default): at large N, where the mesh's node numbering can be cut
 *                          into windows of at most 3200 columns that no element straddles (bodies
 *                          numbered one after the other), the FP32 bulk assembly accumulates each
 *                          row window by window in shared memory; 0: the rows accumulate in A
 *   "mixed.reassembly_group" flagged wavenumbers re-assembled and refined together (1..32,
 *                          default 32; device memory may lower it)
 *   "mixed.reassembly"     system of the flagged wavenumbers: 1 (default) bulk pairs in float-float
 *                          (~48-bit, FP32 pipes), 0 in FP64; near pairs and diagonal are FP64
 *   "assemble.bulk_ff"     bie_assemble's bulk pairs in float-float (1) or FP64 (0, default)
 *   "mixed.graph"          1: replay the device work of full batches from a captured CUDA graph
 *                          (default), 0: launch every kernel directly
 *   "mixed.phase_timing"   1: time the phases of each call with CUDA events (see
 *                          bie_get_phase_times; graphs are then not used), 0: off (default)
 * Learned warm start and Krylov solve (BIE_MODE_LEARNED):
 *   "learned.stride"       every stride-th wavenumber of the call is an anchor (>= 2, default 8;
 *                          indices stride-1, 2 stride-1, ...; the last index if none)
 *   "learned.x0"           initial guess of the GMRES solves: 1 the network (default), 0 zero,
 *                          2 the nearest anchor's solution, 3 the bracketing anchors' solutions
 *                          demodulated by exp(-i k_a d.x), interpolated linearly in k and
 *                          modulated with exp(i k d.x)
 *   "learned.epochs"       training epochs (0..100000, default 60)
 *   "learned.batch"        rows per minibatch (128..1048576, rounded up to 128; default 8192)
 *   "learned.lr", "learned.lr_min"  Adam step size, cosine-decayed to lr_min (default 2e-3, 1e-4)
 *   "learned.seed"         initial weights and minibatch order (default 1234)
 *   "learned.kmax"         wavenumber scale of the feature map (0: the largest training k)
 *   "learned.graph"        1: replay each training epoch from a captured CUDA graph (default)
 *   "gmres.m"              Arnoldi steps per cycle (1..62, default 30)
 *   "gmres.cycles"         cycles, each from a float-float residual (1..100, default 3)
 *   "gmres.inner_tol"      relative residual decrease that ends a cycle (default 1e-5)
 * The refinement target "refine.tol" is also the GMRES backward-error target.
 * Errors: INVALID_ARG for an unknown name or a value out of range. */
int bie_set_option(bie_ctx* ctx, const char* name, double value);

/* Assembles the FP64 system of one wavenumber k >= 0: Eq. (BRIEF) at every node with the App. B
 * term 4 pi P(x_i), unknown P at hard nodes and dP/dn at soft nodes, known values from the
 * scattered-field boundary conditions of Sec. 4 (p_scat = -p_inc soft, dp_scat/dn = -dp_inc/dn
 * hard) moved to the right-hand side.  k = 0 is the zero-frequency term of Eq. (inverseFourier): the
 * kernels take their k -> 0 limit (G = 1/R, g = 1, f = nu_i.(x - x_i)), the Laplace problem.
 *   A_out device c128 [N][N] row-major, b_out device c128 [N].
 * Errors: INVALID_ARG (k < 0, 0 < k < 1e-30 or not finite, NULL pointer), STATE (no geometry). */
int bie_assemble(bie_ctx* ctx, double k, void* A_out, void* b_out);

/* Frequency solves (the per-k hot path): for each k[m] assemble, factor and solve.
 *   k        host f64 [Nk]: each 0 (the zero-frequency term, solved by the k -> 0 limit of the
 *            same kernels, see bie_assemble; not in BIE_MODE_LEARNED) or >= 1e-30
 *   mode     BIE_MODE_FP64, BIE_MODE_MIXED or BIE_MODE_LEARNED (which trains the context's
 *            network on this call's anchors, replacing its parameters)
 *   surf_out device c128 [Nk][2][N]: scattered P and dP/dn at every node, per k
 *   rep      host bie_report [Nk] or NULL
 * Synchronises the stream before returning (the reports are read back).  Errors: INVALID_ARG,
 * STATE, OOM (scratch larger than free device memory), CUDA, TIMEOUT (a bounded wait of the
 * tensor-core factorisation or of a cooperative panel gave up: that factor is void). */
int bie_solve_frequencies(bie_ctx* ctx, const double* k, int64_t Nk, int mode, void* surf_out,
                          bie_report* rep);

/* The mixed-precision frequency solves of bie_solve_frequencies (Sec. 3 Eq. BRIEF assembled,
 * factored and solved per wavenumber as in Sec. 4), stream-ordered: the call returns once its work
 * is enqueued on the context's stream, so that host work and other contexts' streams overlap it.
 * Every decision the synchronous call takes on the host runs on the device instead: wavenumbers
 * flagged by their refinement state or sensitivity estimate are re-assembled in FP64 and refined
 * against that system with their own TF32 factor, in rounds over the batch's flagged systems.
 *   k        host f64 [Nk], as bie_solve_frequencies; copied into the launches, free on return
 *   mode     BIE_MODE_MIXED
 *   surf_out device c128 [Nk][2][N], written in stream order
 *   rep      host bie_report [Nk] or NULL: filled by a host function in stream order, valid once
 *            the stream has completed this call's work (e.g. after cudaStreamSynchronize); the
 *            array must stay allocated until then
 * Differences from bie_solve_frequencies: no last-resort full FP64 solve -- a wavenumber whose
 * re-assembly does not converge, or whose factor met a zero pivot, keeps BIE_FLAG_NOT_CONVERGED
 * (so does every system of a batch whose factorisation gave up a bounded wait, backward error NaN;
 * bie_solve_frequencies on those wavenumbers takes the remaining steps);
 * "mixed.graph" and "mixed.phase_timing" do not apply.  The first solve after bie_set_geometry
 * builds the mixed path's geometry tables and may synchronise.  Calls on one context share its
 * workspace and are ordered by its stream.  Errors (before anything is enqueued): as
 * bie_solve_frequencies; INVALID_ARG for another mode or linear elements. */
int bie_solve_frequencies_async(bie_ctx* ctx, const double* k, int64_t Nk, int mode, void* surf_out,
                                bie_report* rep);

/* Frequency solves for several incident plane waves at once (Sec. 5: for a fixed configuration the
 * solution matrix is kept and only the incident wave changes).  Per wavenumber the system matrix
 * is assembled and factored once; the right-hand side of direction d is -B known_d, B the
 * known-column matrix (the coefficients of the known boundary values in Eq. BRIEF, i.e. the system
 * matrix with every node's condition exchanged, assembled once by the same kernels), known_d the
 * scattered-field boundary values of exp(i k d.x) (Sec. 4).
 *   k        host f64 [Nk] as bie_solve_frequencies
 *   dirs     host f64 [ndir][3], non-zero (normalised here); the context's own direction is unused
 *   mode     BIE_MODE_FP64 or BIE_MODE_MIXED (iterative refinement per direction against the shared
 *            factor; flagged wavenumbers re-assembled per direction as in bie_solve_frequencies)
 *   surf_out device c128 [Nk][ndir][2][N]: P and dP/dn per wavenumber and direction
 *   rep      host bie_report [Nk][ndir] or NULL
 * Memory: one more N x N matrix per wavenumber in flight than bie_solve_frequencies.
 * Synchronises.  Errors: as bie_solve_frequencies; INVALID_ARG for ndir outside [1, 4096], a zero
 * direction or BIE_MODE_LEARNED. */
int bie_solve_frequencies_multi(bie_ctx* ctx, const double* k, int64_t Nk, const double* dirs, int64_t ndir,
                                int mode, void* surf_out, bie_report* rep);

/* Scattered field at M observation points (Eq. BRIEFdmn with the closest surface point x0 of
 * each point, Sec. 3), for every k:
 *   xobs  device f64 [M][3] points in the fluid (a point behind its closest surface point, i.e.
 *         inside a body, is rejected with INVALID_ARG naming the lowest such index)
 *   k     host f64 [Nk] (k = 0 allowed, as in bie_solve_frequencies); surf device c128 [Nk][2][N]
 *         as written by bie_solve_frequencies
 *   T_out device c128 [Nk][M]
 *   mode  BIE_MODE_FP64 (FP64 arithmetic) or BIE_MODE_MIXED (FP32 with float-float phases)
 * Foot points are computed on the device at every call (the inside test reads one word back).
 * Errors: INVALID_ARG, STATE, CUDA. */
int bie_eval_field(bie_ctx* ctx, const double* xobs, int64_t M, const double* k, int64_t Nk,
                   const void* surf, int mode, void* T_out);

/* Spectra of sampled pulses with the sign of Eq. (inverseFourier):
 *   S[p][m] = sum_n s[p][n] exp(+2 pi i m n / Nt), m = 0 .. Nt/2.
 *   s device f64 [P][Nt], S_out device c128 [P][Nt/2+1].  Nt a power of two in [2, 4096]. */
int bie_pulse_spectrum(bie_ctx* ctx, const double* s, int64_t P, int64_t Nt, void* S_out);

/* Space-time scattered field (Sec. 3 end, Sec. 4): for each pulse p, point x and time sample n
 *   out[p][x][n] = (1/Nt) sum_r w_m Re( S[p][m] T[r][x] exp(-2 pi i m n / Nt) ),  m = midx[r],
 * w_m = 1 for m = 0 or Nt/2, else 2 (real signals); frequencies not listed contribute zero.
 *   T device c128 [Nk][M]; midx host i64 [Nk], strictly increasing, 0 <= m <= Nt/2
 *   S device c128 [P][Nt/2+1]; out device, f64 (out_dtype 0) or f32 (out_dtype 1), [P][M][Nt]
 * Errors: INVALID_ARG (sizes, ordering, Nt not a power of two in [2, 4096]). */
int bie_synthesize(bie_ctx* ctx, const void* T, const int64_t* midx, int64_t Nk, int64_t M,
                   const void* S, int64_t P, int64_t Nt, void* out, int out_dtype);

/* Dominant frequencies of the incident pulses (Sec. 4, Table I, and Sec. 5: accurate space-time
 * fields follow from the few wavenumbers at which the incident spectrum is largest, so only those
 * need a frequency solve).  Ranks m = 0 .. Nt/2 by max over the pulses of |S[p][m]| (ties: the
 * lower m first) and returns the K largest in ascending order, ready as bie_synthesize's midx
 * (the wavenumbers to solve are k_m = 2 pi m / (c T) for the window length T).
 *   S device c128 [P][Nt/2+1] as written by bie_pulse_spectrum; midx_out host i64 [K].
 * Synchronises.  Errors: INVALID_ARG (P < 1, Nt not a power of two in [2, 4096], K outside
 * [0, Nt/2 + 1], NULL pointer). */
int bie_top_frequencies(bie_ctx* ctx, const void* S, int64_t P, int64_t Nt, int64_t K, int64_t* midx_out);

/* Allocation-free variant of bie_synthesize.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory while they run -- a host framework that
 * hands out a fixed device-memory budget through its own pool, or a latency-bound pipeline in
 * which cudaMalloc/cudaFree would synchronise the device.  It needs no context and allocates
 * nothing: its scratch (the FFT twiddle table and the device copy of midx) lives in one
 * file-scope device array of 64 KB that every GPU loading the library holds until the process
 * exits.  Arguments and the result are those of bie_synthesize, on the caller's current device
 * and on `stream` (a cudaStream_t, NULL = legacy default stream); the call returns after the
 * stream has completed.
 * Limits: Nt a power of two in [2, 4096] and Nk <= 4096 (midx entries are in [0, Nt/2] anyway);
 * larger sizes return BIE_ERR_INVALID_ARG with a message.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) and keeps it for the process; make that first
 * call before any stream capture begins, and do not use this entry point after a cudaDeviceReset
 * of that device (the kept address would be stale).  All calls share the one array and every call rewrites the parts it uses, so
 * calls whose work overlaps on the GPU (different streams or threads) race. */
int bie_synthesize_noalloc(const void* T, const int64_t* midx, int64_t Nk, int64_t M, const void* S,
                           int64_t P, int64_t Nt, void* out, int out_dtype, void* stream);

/* Device time of each phase of the last BIE_MODE_MIXED call, recorded when the option
 * "mixed.phase_timing" was 1 (the call then launches every kernel directly instead of replaying
 * captured graphs).  out host.  Not part of the paper's method: a measurement aid for the
 * rooflines of the factorisation and assembly. */
int bie_get_phase_times(bie_ctx* ctx, bie_phase_times* out);

/* Micro-benchmarks of the pipes that bound the library's kernels on device `cuda_device`: FP32
 * and FP64 FMA throughput (CUDA cores) and dense tcgen05 tensor-core throughput for TF32 and BF16
 * operands (M = 128, N = 256 MMAs issued back to back from shared memory, one CTA per SM).  Each
 * rate is the best of five timed launches (CUDA events), a few milliseconds each; the call
 * allocates 256 bytes and synchronises.  Not part of the paper's method: the denominators of the
 * roofline fractions.  Errors: INVALID_ARG (device), CUDA, TIMEOUT (a bounded wait gave up). */
int bie_measure_peaks(int cuda_device, bie_peaks* out);

/* Autotuner of the mixed path (not part of the paper's method, which fixes no launch parameters):
 * for the context's geometry, times one batch of BIE_MODE_MIXED solves (sample wavenumbers
 * k host f64 [nk], repeated to fill the batch) for every candidate of "mixed.batch" in
 * {8, 16, 32, 64, 128, 256} that fits a third of free device memory and "mixed.tcgen05" in {3, 2}
 * (with "mixed.lu_block" 256), then, if version 3 won, "mixed.lu_block" 128 and 512 at the chosen
 * batch, then "mixed.lu_panel" 32 at the chosen batch and block, then "mixed.lu_tile" 128, and
 * sets the fastest per wavenumber on the context.  cache_path (host string or NULL): a JSON
 * file keyed by N rounded up to 64; an entry for this N is applied without measuring, a new
 * measurement is added to it.  out (host, optional) receives the choice.  Synchronises.
 * Errors: STATE without geometry, OOM if no candidate fits, INVALID_ARG if the cache cannot be
 * written. */
int bie_autotune(bie_ctx* ctx, const double* k, int64_t nk, const char* cache_path, bie_tune_result* out);

/* Scheduler of many independent jobs (scatterer configurations, each with its own mesh and
 * wavenumber list) on one GPU: jobs run largest-first on `workers` threads, each with its own
 * context and CUDA stream, so that small configurations overlap large ones.  tune_cache (host
 * string or NULL): autotuner cache applied to every job's N bucket (measured on first use).
 * Not part of the paper's method.  Errors: INVALID_ARG (device, workers outside [1, 64]). */
int bie_sched_create(bie_sched** out, int cuda_device, int workers, const char* tune_cache);
int bie_sched_destroy(bie_sched* sched);
/* Queues a job.  Mesh arguments as bie_set_geometry (copied now), dir as
 * bie_set_incident_plane_wave (NULL: +z), k host f64 [Nk] (copied), mode and outputs as
 * bie_solve_frequencies: surf_out device c128 [Nk][2][N] and rep host [Nk] (or NULL), both
 * written during bie_sched_run.  job_id (optional) receives the job's index. */
int bie_sched_add(bie_sched* sched, const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                  const double* normals, const uint8_t* bc, const double* dir, const double* k, int64_t Nk,
                  int mode, void* surf_out, bie_report* rep, int32_t* job_id);
/* Runs every queued job and returns when all are done (the queue is then empty).  stats (host,
 * optional).  Errors: the first failing job's code, with its message. */
int bie_sched_run(bie_sched* sched, bie_sched_stats* stats);

/* ---- learned warm start (BIE_MODE_LEARNED's network; not part of the paper's method) ---------
 * Feature map of node x (normal nu) at wavenumber k, 64 values: (x - c)/s, nu, k/kmax, (k/kmax)^2,
 * then cos and sin of k * sc_q * (b_j . (x - c)) for j = 0..6, q = 0..3 (value 8 + 2(4j+q) is the
 * cosine, 9 + 2(4j+q) the sine), b = {d, e_x, e_y, e_z, (e_x+e_y)/sqrt2, (e_y+e_z)/sqrt2,
 * (e_z+e_x)/sqrt2}, sc = {0.5, 1, 1.5, 2}; c = centroid of the nodes, s = largest node distance
 * from c, kmax = "learned.kmax" or the largest wavenumber of the last training.
 * Network: h1 = tanh(W1 phi + b1), h2 = tanh(W2 h1 + b2), h3 = tanh(W3 h2 + b3), y = W4 h3 + b4;
 * parameters (FP32) in the order W1 [256][64], b1 [256], W2 [256][256], b2, W3 [256][256], b3,
 * W4 [2][256], b4 [2] (row-major, BIE_MLP_PARAMS values).  Hidden layers run with BF16 operands
 * and FP32 accumulation on the tensor cores.  Loss over B rows: (1/B) sum |y - t|^2.
 * Targets when training on solutions: t = u exp(-i k d.x) / tau, u the node's unknown (P at
 * hard, dP/dn at soft nodes), tau the root mean square of |u| over the training rows; the
 * prediction is x0 = tau (y0 + i y1) exp(i k d.x). */

/* Copies in (host f32 [BIE_MLP_PARAMS]) the network parameters and resets the optimiser. */
int bie_mlp_set_params(bie_ctx* ctx, const float* theta);
/* Copies out (host f32 [BIE_MLP_PARAMS]).  Errors: STATE before any parameters exist. */
int bie_mlp_get_params(bie_ctx* ctx, float* theta);
/* Features of every node at k[0..nk) (host f64), as fed to the network (rounded to BF16):
 * phi_out device f32 [nk][N][64].  Errors: STATE without geometry or wavenumber scale. */
int bie_mlp_features(bie_ctx* ctx, const double* k, int64_t nk, float* phi_out);
/* Network outputs: X device f32 [B][64], Y_out device f32 [B][2].  Synchronises. */
int bie_mlp_forward(bie_ctx* ctx, const float* X, int64_t B, float* Y_out);
/* Loss and its gradient: X device f32 [B][64], T device f32 [B][2]; grad_out device f32
 * [BIE_MLP_PARAMS], loss_out device f32 [1] (either may be NULL).  Synchronises. */
int bie_mlp_loss_grad(bie_ctx* ctx, const float* X, const float* T, int64_t B, float* grad_out,
                      float* loss_out);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected, step size lr) with the
 * gradient grad (device f32 [BIE_MLP_PARAMS]) on the context's parameters and moments. */
int bie_mlp_adam_step(bie_ctx* ctx, const float* grad, double lr);
/* Trains on surface solutions: k host f64 [nk], surf device c128 [nk][2][N] (as written by
 * bie_solve_frequencies); runs `epochs` epochs with the "learned.*" options, starting from the
 * current parameters (or a seeded Glorot initialisation).  loss_hist host f32 [epochs] or NULL. */
int bie_mlp_train(bie_ctx* ctx, const double* k, int64_t nk, const void* surf, int epochs,
                  float* loss_hist);
/* Predicted unknowns x0 = tau (y0 + i y1) exp(i k d.x) at every node: k host f64 [nk], x0_out
 * device c128 [nk][N].  Synchronises. */
int bie_mlp_predict(bie_ctx* ctx, const double* k, int64_t nk, void* x0_out);
/* Summary of the last BIE_MODE_LEARNED solve (host out). */
int bie_get_learned_info(bie_ctx* ctx, bie_learned_info* out);

#ifdef __cplusplus
}
#endif
#endif
