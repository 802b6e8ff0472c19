// bie_common.cuh -- internal types and device helpers shared by the library's translation units.
// Not part of the public interface (include/bie.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/bie.h"

namespace bie {

constexpr double kPi = 3.141592653589793238462643383279502884;

// ------------------------------------------------------------------------------------------
// Error plumbing: every entry point funnels failures through set_error() and returns a code.
// ------------------------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define BIE_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return ::bie::cuda_fail(_e, #expr); \
  } while (0)

// Every kernel launch of the library goes through BIE_LAUNCH, which counts it (bie_kernel_launches).
void count_launch();
void count_launches(int64_t n);
void uncount_launches(int64_t n);
#define BIE_LAUNCH(...) (::bie::count_launch(), __VA_ARGS__)

#define BIE_TRY(expr)          \
  do {                         \
    int _rc = (expr);          \
    if (_rc != BIE_OK) return _rc; \
  } while (0)

// ------------------------------------------------------------------------------------------
// Quadrature tables (host-built, uploaded once per geometry).
// Standard rule: Q points per element.  Near rule for local node a: nnear[a] points, stored
// with stride QN (= 2 * ng_near^2) per (element, local node).
// ------------------------------------------------------------------------------------------
struct QuadRule {
  int ng = 4, ng_near = 6;
  int Q = 0, QN = 0;
  int nnear[6] = {0, 0, 0, 0, 0, 0};
  std::vector<double> xi, eta, w;           // [Q]
  std::vector<double> nxi, neta, nw;        // [6][QN]
};
void build_quad_rule(QuadRule& r, int ng, int ng_near);
void gauss_legendre_unit(int n, double* x, double* w);

// Per-point geometry record layout in the device tables (structure of arrays, FP64):
// x, y, z, nx, ny, nz, wJ  -> 7 arrays of length npts.
enum { GX = 0, GY, GZ, GNX, GNY, GNZ, GWJ, GCOUNT };

// ------------------------------------------------------------------------------------------
// The context.
// ------------------------------------------------------------------------------------------
struct DeviceBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct MlpState;  // learned warm start (mlp.cu)

// Per-system state of the iterative refinement and of the Krylov solver's outer loop.
struct RefineState {
  int32_t done;      // 1 once converged
  int32_t iters;     // corrections applied (refinement) or Arnoldi steps (Krylov)
  double anorm;      // ||A||_inf
  double bnorm;      // ||b||_inf
  double berr;       // latest backward error
  double err_est;    // estimated relative error caused by FP32 assembly (see refine.cu, k_perturb)
  double scale;      // ||A||_inf ||x||_inf + ||b||_inf at the latest check
};

}  // namespace bie

struct bie_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int ng = 4, ng_near = 6;
  double dir[3] = {0.0, 0.0, 1.0};

  // geometry (device)
  bool has_geom = false;
  int64_t N = 0, E = 0;
  double* nodes = nullptr;     // [N][3]
  int32_t* elems = nullptr;    // [E][6]
  double* normals = nullptr;   // [N][3]
  uint8_t* bc = nullptr;       // [N]
  uint8_t* bc_flip = nullptr;  // [N] 1 - bc: assembles the known-column matrix (several directions)
  // linear 3-node elements (bie_set_geometry_linear): the geometry above is their flat quadratic
  // image (N = lin_N vertices, then one mid-edge node per edge); 0 for quadratic meshes
  int64_t lin_N = 0;
  int32_t* lin_adj_off = nullptr;  // [lin_N + 1] CSR: mid-edge nodes next to each vertex
  int32_t* lin_adj = nullptr;
  int32_t* lin_mid = nullptr;      // [2][N - lin_N] the two vertices of each mid-edge node
  std::vector<double> h_nodes, h_normals;
  std::vector<int32_t> h_elems;
  std::vector<uint8_t> h_bc;
  bie::QuadRule rule;
  double* qgeo = nullptr;      // standard points: GCOUNT x [E*Q]
  double* ngeo = nullptr;      // near points:     GCOUNT x [E*6*QN]
  double* qshape = nullptr;    // [Q][6] shape values at the standard points
  double* nshape = nullptr;    // [6][QN][6] shape values at the near points
  float* nshape32 = nullptr;   // the same in FP32 (mixed path)
  float* qgeo32 = nullptr;     // mixed path standard points: see asm32.cu for the layout
  float* qshape32 = nullptr;   // [Q][6]
  int ncolors = 0;
  std::vector<int32_t> h_color_off;  // [ncolors+1]
  int32_t* color_off = nullptr;
  int32_t* elem_perm = nullptr;      // [E] elements ordered by colour, then by column window
  // column windows: node ranges [win_lo[w], win_lo[w + 1]) of at most kWinMax nodes that no element
  // straddles (0: no such partition; 1: one window, all of [0, N)); within colour col the
  // elements of window w are [wcol_off[col (nwin + 1) + w], wcol_off[col (nwin + 1) + w + 1])
  int nwin = 0, win_max = 0;
  int32_t* win_lo = nullptr;         // [nwin + 1]
  int32_t* wcol_off = nullptr;       // [ncolors][nwin + 1]
  int32_t* n2e_off = nullptr;        // [N+1] CSR: elements containing node i
  int32_t* n2e = nullptr;            // element * 8 + local index
  int max_n2e = 0;
  double far_r2 = 0.0;               // (3 x longest element edge)^2, set on first mixed assembly
  int* d_nnear = nullptr;            // [6] near-rule point counts

  // mixed-precision path settings
  int tc_version = 3;                // LU trailing update: 0 SIMT FP32, 1 tcgen05 (register-staged),
                                     // 2 tcgen05 (persistent, TMA-fed, warp-specialised), 3 as 2
                                     // with the update deferred over 256-column blocks
  int lu_block = 0;                  // mixed.tcgen05 3: columns over which the trailing update is
                                     // deferred (128, 256 or 512; 0: 512 from N = 8192 on, else 256)
  int lu_coop = 1;                   // several CTAs per matrix in the panels of few tall matrices
  int lu_panel = 64;                 // mixed.tcgen05 3: panel width (32 or 64)
  int lu_tile = 256;                 // mixed.tcgen05 2, 3: update tile width in real columns (256 or 128)
  int mixed_batch = 256;             // wavenumbers per batch (capped by free memory; the tuner's
                                     // choice at N = 2884)
  int refine_it_max = 10;            // refinement corrections per system
  int refine64_it_max = 30;          // corrections against the FP64 re-assembly of flagged systems
  double refine64_tol = 1e-13;       // backward-error target against the FP64 re-assembly
  double refine_tol = 1e-11;         // backward-error target of the refinement
  double fallback_err_est = 3e-7;    // FP64 re-solve above this estimated assembly-induced error (the
                                     // true error is 0.14 - 4.4 times the estimate on the two-sphere
                                     // sweep; at 3e-7 the largest unflagged error there is 4.5e-7)
  int field_accurate_phase = 1;      // mixed field: float-float phases (1) or FP32 phases (0)
  int field_variant = 2;             // mixed field kernel: 2 k_field32c (16 wavenumbers per group,
                                     // 128 points per CTA, 32-point tiles), 1 the same with 64
                                     // points and 64-point tiles, 0 k_field32b (8 per group)
  int assemble_ff = 0;               // bie_assemble: bulk pairs in float-float (1) or FP64 (0)
  int uniform_bc = -1;               // every element has one condition on all nodes (1), not (0), unknown
  int asm_kb = 2;                    // FP32 bulk assembly: wavenumbers per thread (1, 2), 0 = the
                                     // general kernel (also taken when an element mixes conditions)
  int asm_windows = 1;               // FP32 bulk assembly at large N: column windows in shared memory (1) or rows in A (0)
  int refactor32 = 1;                // before the full FP64 path: FP32 re-factorisation of the FP64 system (1)
  int reassembly_group = 32;         // FP64 re-assembly slots refined together (1..32; memory may lower it)
  int reassembly_ff = 1;             // flagged wavenumbers: bulk re-assembly in float-float (1) or FP64 (0)
  int mixed_graph = 1;               // replay full batches of the mixed path from a CUDA graph
  int phase_timing = 0;              // time the mixed path's phases with CUDA events (no graphs)
  size_t mem_budget = 0;             // device bytes this context may size its workspaces to
                                     // (0: all free memory; the scheduler gives each worker a share)
  bie_phase_times phase{};           // phases of the last BIE_MODE_MIXED call (phase_timing 1)
  void* pinned = nullptr;            // pinned host staging (wavenumbers of graph replays)
  cudaStream_t cap_stream = nullptr; // private stream on which CUDA graphs are captured
  size_t pinned_bytes = 0;
  void* rep_pinned = nullptr;        // pinned staging of the stream-ordered solves' reports
  size_t rep_pinned_bytes = 0;
  std::vector<void*> rep_pinned_old; // outgrown report staging (an earlier call may still use it)

  // learned warm start + Krylov path (BIE_MODE_LEARNED)
  int learned_stride = 8;            // every stride-th wavenumber is solved directly (an anchor)
  int learned_x0 = 1;                // initial guess: 0 zero, 1 network, 2 nearest anchor's solution
  int mlp_epochs = 60;               // training epochs over the anchors' solutions
  int mlp_batch = 8192;              // rows per minibatch
  double mlp_lr = 2e-3, mlp_lr_min = 1e-4;  // Adam step size, cosine-decayed to lr_min
  int64_t mlp_seed = 1234;           // initial weights and minibatch order
  double mlp_kmax = 0.0;             // feature wavenumber scale (0: largest training wavenumber)
  int mlp_graph = 1;                 // replay training epochs from a captured CUDA graph
  int gmres_m = 30;                  // Arnoldi steps per cycle
  int gmres_cycles = 3;              // cycles (each starts from a float-float residual)
  double gmres_inner_tol = 1e-5;     // relative residual decrease that closes a cycle
  bie::MlpState* mlp = nullptr;
  bie_learned_info learned_info{};

  // workspace (device), grown on demand
  bie::DeviceBuf work;   // per-call systems / factors
  bie::DeviceBuf work2;  // FFT twiddles
  bie::DeviceBuf work3;  // foot points, field scratch, synthesis indices
  bie::DeviceBuf work4;  // learned mode: the anchors' factors, permutations and solutions
  bie::DeviceBuf work5;  // linear elements: surface values interpolated onto the flat quadratic image
  bie::DeviceBuf work6;  // float-float re-assembly: known values split into float-float
};

namespace bie {

// Device memory of a context comes from the stream-ordered allocator on the context's stream
// (cudaMallocAsync / cudaFreeAsync): freeing and growing buffers never synchronises the device,
// so contexts on other streams (the scheduler's workers) keep running.
int dev_alloc(bie_ctx* c, void** p, size_t bytes);
void dev_free(bie_ctx* c, void* p);
int ensure_buf(bie_ctx* c, DeviceBuf& b, size_t bytes);
// Free device memory for this context's workspace sizing: cudaMemGetInfo, capped by mem_budget.
int device_free(bie_ctx* c, size_t* free_b);
// The device's per-block shared-memory opt-in limit.  Kernels with dynamic shared memory get
// this limit once (never a launch-specific size), so that contexts on other threads launching
// the same kernel with other sizes cannot lower it between another thread's set and launch.
int smem_optin();
template <typename F>
inline int set_smem_max(F* f) {  // dynamic limit = opt-in limit minus the kernel's static shared memory
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, (const void*)f) != cudaSuccess) return fail(BIE_ERR_CUDA, "cudaFuncGetAttributes");
  const cudaError_t e = cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem_optin() - (int)a.sharedSizeBytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(MaxDynamicSharedMemorySize)");
  return BIE_OK;
}
// Graph capture: work enqueued on c->stream between begin and end is recorded (not run) on the
// context's private capture stream -- the caller's stream may be the legacy default stream, which
// cannot be captured -- and returned as a graph to be launched on c->stream.
int capture_begin(bie_ctx* c, cudaStream_t* saved);
int capture_end(bie_ctx* c, cudaStream_t saved, cudaGraph_t* graph);
int ensure_pinned(bie_ctx* c, size_t bytes);
void free_buf(DeviceBuf& b);

// ------------------------------------------------------------------------------------------
// Device helpers.
// ------------------------------------------------------------------------------------------
struct cd {  // complex double
  double re, im;
};
struct cf {  // complex float
  float re, im;
};

__host__ __device__ __forceinline__ cd cmul(cd a, cd b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ cd cadd(cd a, cd b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ cd csub(cd a, cd b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ cd cscale(cd a, double s) { return {a.re * s, a.im * s}; }

// ---- float-float ("double-float") arithmetic: value = hi + lo, |lo| <= ulp(hi)/2 ----------
// Error-free transforms after Knuth (TwoSum) and Dekker/FMA (TwoProd); renormalisation by
// Fast2Sum.  About 48 significant bits.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, err};
}
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = ff_two_sum(a.hi, b.hi);
  float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return ff_fast_two_sum(s.hi, lo);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_sqr(ff a) {
  float p = __fmul_rn(a.hi, a.hi);
  float e = __fmaf_rn(a.hi, a.hi, -p);
  e = __fmaf_rn(2.0f * a.hi, a.lo, e);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_sqrt(ff a) {  // a > 0
  float y = sqrtf(a.hi);
  float r = __fmaf_rn(-y, y, a.hi);  // exact residual of y^2 vs a.hi
  r = __fadd_rn(r, a.lo);
  return ff_fast_two_sum(y, __fdividef(r, 2.0f * y));
}
// ---- float-float geometry with lazy tails -------------------------------------------------
// Distances and projections for the FP32 kernels' phases keep head + tail as an unevaluated sum
// without renormalising it: a tail may reach a few ulp of the coordinates (a difference of
// nearby points), and every consumer (error-free products, cis_ffprod, the square root below)
// takes head and tail as they are.  Relative errors: about 2e-11 on R, 1 ulp on 1/R.
__device__ __forceinline__ ff ff_diff_lazy(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, -b.hi);
  return {s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo))};
}
// x^2 + y^2 + z^2: the heads' squares error-free (FMA), their sum by two error-free additions,
// and the errors with the tails' terms 2 hi lo + lo^2 gathered into the tail.
__device__ __forceinline__ ff ff_norm2_lazy(ff x, ff y, ff z) {
  const float px = __fmul_rn(x.hi, x.hi), py = __fmul_rn(y.hi, y.hi), pz = __fmul_rn(z.hi, z.hi);
  float ex = __fmaf_rn(x.hi, x.hi, -px), ey = __fmaf_rn(y.hi, y.hi, -py), ez = __fmaf_rn(z.hi, z.hi, -pz);
  ex = __fmaf_rn(x.lo, x.lo, __fmaf_rn(x.hi + x.hi, x.lo, ex));
  ey = __fmaf_rn(y.lo, y.lo, __fmaf_rn(y.hi + y.hi, y.lo, ey));
  ez = __fmaf_rn(z.lo, z.lo, __fmaf_rn(z.hi + z.hi, z.lo, ez));
  const ff s1 = ff_two_sum(px, py), s2 = ff_two_sum(s1.hi, pz);
  return {s2.hi, __fadd_rn(__fadd_rn(__fadd_rn(ex, ey), ez), __fadd_rn(s1.lo, s2.lo))};
}
// a . (x, y, z) for a float-float vector a: error-free head products (FMA, with the cross
// terms), two error-free additions, errors gathered into the tail.
__device__ __forceinline__ ff ff_dot3_lazy(const ff* a, ff x, ff y, ff z) {
  const float p0 = __fmul_rn(a[0].hi, x.hi), p1 = __fmul_rn(a[1].hi, y.hi), p2 = __fmul_rn(a[2].hi, z.hi);
  float e0 = __fmaf_rn(a[0].hi, x.hi, -p0), e1 = __fmaf_rn(a[1].hi, y.hi, -p1), e2 = __fmaf_rn(a[2].hi, z.hi, -p2);
  e0 = __fmaf_rn(a[0].hi, x.lo, __fmaf_rn(a[0].lo, x.hi, e0));
  e1 = __fmaf_rn(a[1].hi, y.lo, __fmaf_rn(a[1].lo, y.hi, e1));
  e2 = __fmaf_rn(a[2].hi, z.lo, __fmaf_rn(a[2].lo, z.hi, e2));
  const ff s1 = ff_two_sum(p0, p1), s2 = ff_two_sum(s1.hi, p2);
  return {s2.hi, __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), e2), __fadd_rn(s1.lo, s2.lo))};
}
// R = sqrt(a) and inv = 1/R for a float-float a > 0 (a lazy tail): y0 = rsqrt(fl(a.hi + a.lo))
// (2 ulp), R.hi = fl(a) y0, R.lo = ((a.hi - R.hi^2) + a.lo) y0 / 2 (the residual by FMA: one
// Newton step, error about y0's squared), inv = y0 + y0 (1 - R.hi y0) / 2 (one Newton step).
__device__ __forceinline__ ff ff_sqrt_lazy(ff a, float& inv) {
  const float s = __fadd_rn(a.hi, a.lo);
  const float y0 = rsqrtf(s);
  const float y = __fmul_rn(s, y0);
  const float h = 0.5f * y0;
  inv = __fmaf_rn(h, __fmaf_rn(-y, y0, 1.0f), y0);
  return {y, __fmul_rn(__fadd_rn(__fmaf_rn(-y, y, a.hi), a.lo), h)};
}

__host__ __device__ __forceinline__ ff ff_from_double(double x) {
  float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}
__host__ __device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// 1/k for the FP32 kernels' f = sin(k nu.r)/k; 0 at k = 0, where f takes its limit nu.r (the
// zero-frequency term): every FP32 kernel forms f = kinv != 0 ? sin(k nu.r) kinv : nu.r.
__host__ __device__ __forceinline__ float kinv32(double k) { return k > 0.0 ? (float)(1.0 / k) : 0.f; }

// cos and sin of v = vh + vl, |v| <= pi (plus rounding), to about FP32 rounding: quadrant
// reduction q = rint(v 2/pi) with pi/2 split in two floats (Cody-Waite), then the Taylor series
// of sin (through v^9) and cos (through v^10) on |v'| <= pi/4, whose truncation errors are below
// 2e-9 and 2e-10; the quadrant selects and negates.  Written from the series, not from a
// library's polynomial.
// Nearest integer (ties to even) of an FP32 value of magnitude below 2^22, as two additions of
// 1.5 * 2^23 on the FMA pipe instead of an instruction of the conversion unit; the sum's low
// significand bits hold that integer modulo 2^22 (two's complement for negative values).
constexpr float kRoundMagic = 12582912.0f;  // 1.5 * 2^23
__device__ __forceinline__ float round_small(float x) {
  return __fsub_rn(__fadd_rn(x, kRoundMagic), kRoundMagic);
}

__device__ __forceinline__ void cis_reduced(float vh, float vl, float& c, float& s) {
  const float kTwoOverPi = 0.636619772367581343f;
  const float kPio2Hi = 1.57079637050628662f;        // fl32(pi/2)
  const float kPio2Lo = -4.37113900018624284e-8f;    // pi/2 - fl32(pi/2)
  const float qm = __fadd_rn(__fmul_rn(vh, kTwoOverPi), kRoundMagic);  // |v 2/pi| < 2^22
  const float q = __fsub_rn(qm, kRoundMagic);
  float v = __fmaf_rn(-q, kPio2Hi, vh);
  v = __fmaf_rn(-q, kPio2Lo, v) + vl;
  const float v2 = v * v;
  float ps = __fmaf_rn(v2, 2.75573192239858907e-6f, -1.98412698412698413e-4f);  // 1/9!, -1/7!
  ps = __fmaf_rn(v2, ps, 8.33333333333333333e-3f);                              // 1/5!
  ps = __fmaf_rn(v2, ps, -1.66666666666666667e-1f);                             // -1/3!
  const float sv = __fmaf_rn(v * v2, ps, v);
  float pc = __fmaf_rn(v2, -2.75573192239858907e-7f, 2.48015873015873016e-5f);  // -1/10!, 1/8!
  pc = __fmaf_rn(v2, pc, -1.38888888888888889e-3f);                             // -1/6!
  pc = __fmaf_rn(v2, pc, 4.16666666666666667e-2f);                              // 1/4!
  pc = __fmaf_rn(v2, pc, -0.5f);
  const float cv = __fmaf_rn(v2, pc, 1.0f);
  const int qi = __float_as_int(qm) & 3;
  const float a = (qi & 1) ? sv : cv, b = (qi & 1) ? cv : sv;
  c = (qi == 1 || qi == 2) ? -a : a;
  s = (qi >= 2) ? -b : b;
}

// pi/2 as an unevaluated sum of three floats: h1 = fl32(pi/2), h2 = fl32(pi/2 - h1),
// h3 = fl32(pi/2 - h1 - h2), from pi to 200 bits; the remainder is below 1.1e-23.
constexpr float kHalfPi1 = 1.57079637050628662f;
constexpr float kHalfPi2 = -4.37113882867379e-8f;
constexpr float kHalfPi3 = -1.71512451000588e-15f;

// e^{i t} for t = p + e, p a float with |p| < 2^20 and e a correction of a few ulp(p) (the tail
// of an error-free product), in one reduction: n = rint(p 2/pi), u = (p - n h1) + (e - n h2 -
// n h3).  The first difference is exact under FMA: for |p| >= 1 both p and n h1 are multiples of
// ulp(h1) = 2^-23 and the difference is below 1; below 1, n is 0 or +-1 and the difference is a
// multiple of ulp(p) below 1.  u then rounds once to FP32 (|u| <= pi/4 plus the quotient's
// rounding), and cos/sin of u come from the Taylor series of cis_reduced, placed in the quadrant
// n mod 4 (read from the low bits of the rounding sum).
__device__ __forceinline__ void cis_split(float p, float e, float& c, float& s) {
  const float kTwoOverPi = 0.636619772367581343f;
  const float qm = __fmaf_rn(p, kTwoOverPi, kRoundMagic);
  const float n = __fsub_rn(qm, kRoundMagic);
  const float h = __fmaf_rn(-n, kHalfPi1, p);
  float t = __fmaf_rn(-n, kHalfPi2, e);
  t = __fmaf_rn(-n, kHalfPi3, t);
  const float v = __fadd_rn(h, t);
  const float v2 = v * v;
  float ps = __fmaf_rn(v2, 2.75573192239858907e-6f, -1.98412698412698413e-4f);  // 1/9!, -1/7!
  ps = __fmaf_rn(v2, ps, 8.33333333333333333e-3f);                              // 1/5!
  ps = __fmaf_rn(v2, ps, -1.66666666666666667e-1f);                             // -1/3!
  const float sv = __fmaf_rn(v * v2, ps, v);
  float pc = __fmaf_rn(v2, -2.75573192239858907e-7f, 2.48015873015873016e-5f);  // -1/10!, 1/8!
  pc = __fmaf_rn(v2, pc, -1.38888888888888889e-3f);                             // -1/6!
  pc = __fmaf_rn(v2, pc, 4.16666666666666667e-2f);                              // 1/4!
  pc = __fmaf_rn(v2, pc, -0.5f);
  const float cv = __fmaf_rn(v2, pc, 1.0f);
  const int qi = __float_as_int(qm) & 3;
  const float a = (qi & 1) ? sv : cv, b = (qi & 1) ? cv : sv;
  c = (qi == 1 || qi == 2) ? -a : a;
  s = (qi >= 2) ? -b : b;
}

// e^{i k R} for float-float k and R (|k R| < 2^20): the product's head and its error-free tail
// (with the cross terms) go to cis_split without renormalisation.
__device__ __forceinline__ void cis_ffprod(ff k, ff R, float& c, float& s) {
  const float p = __fmul_rn(k.hi, R.hi);
  float e = __fmaf_rn(k.hi, R.hi, -p);
  e = __fmaf_rn(k.hi, R.lo, e);
  e = __fmaf_rn(k.lo, R.hi, e);
  cis_split(p, e, c, s);
}

// Barrier of the nthreads threads (whole warps) that use barrier `id` (1..15; 0 is
// __syncthreads); orders their shared- and global-memory accesses like __syncthreads.
__device__ __forceinline__ void bar_named(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Compensated (Kahan-Babuska/Neumaier) running sum in FP32.
struct ksum {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    ff t = ff_two_sum(s, x);
    s = t.hi;
    c = __fadd_rn(c, t.lo);
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

}  // namespace bie
