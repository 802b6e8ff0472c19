// gmres.cu -- restarted flexible GMRES (Saad, 1993) for a batch of frequency systems, right-
// preconditioned by the low-precision LU factor of a nearby wavenumber's system (the "anchor"),
// inside an outer refinement loop:
//   repeat:  r = b - A x  (float-float, as in refine.cu);  stop when the backward error is small;
//            run up to m Arnoldi steps on A M^{-1} from r (FP32 products, FP64 basis) until the
//            residual estimate falls by `inner_tol`;  x += Z y.
// Each system carries its own state on the device; the host enqueues a fixed number of steps per
// cycle and kernels of systems that have finished the cycle (or converged) return at once.
#include "bie_common.cuh"

namespace bie {

__global__ void k_trsv_lu(const cf* __restrict__ LU, int n, int64_t ld, int64_t bstride, const int32_t* __restrict__ perm,
                          const cd* __restrict__ rhs, cd* __restrict__ out, int accumulate,
                          const RefineState* __restrict__ st, const int32_t* __restrict__ sel, int64_t rstride,
                          int64_t roff, int64_t ostride, int64_t ooff, const cf* __restrict__ Dinv, int64_t dstride);
int64_t diag_inv_stride(int n);
int residual_ff(bie_ctx* c, const cf* A, int n, int64_t ld, int64_t bstride, int nk, const cd* b, const cd* x, cd* r,
                double* rowabs, const RefineState* st);
__global__ void k_refine_check(int n, const cd* __restrict__ b, const cd* __restrict__ x, const cd* __restrict__ r,
                               const double* __restrict__ rowabs, RefineState* __restrict__ st, double tol,
                               int count_iter);

struct GmresState {
  int32_t j;        // Arnoldi steps taken in the current cycle
  int32_t iters;    // total Arnoldi steps
  double beta;      // ||r|| at the start of the cycle
  double resid;     // current residual estimate |g_{j}|
  double target;    // absolute residual at which the outer backward-error target is met
};

// ---- block reductions (1024 threads) -------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// start of a cycle: beta = ||r||_2, v_0 = r / beta, g = (beta, 0, ...); gate = converged
// The cycle also stops once |g| falls below target = tol (||A|| ||x|| + ||b||) / 2 (infinity
// norms, from the latest check; |g| bounds the 2-norm and so the infinity norm of the residual):
// a close initial guess then saves the Arnoldi steps of the last decades.
__global__ void __launch_bounds__(1024) k_gm_start(int n, int m, const cd* __restrict__ r, cd* __restrict__ V,
                                                   cd* __restrict__ g, GmresState* __restrict__ gs,
                                                   const RefineState* __restrict__ rs, RefineState* __restrict__ gate,
                                                   double tol) {
  __shared__ double red[32];
  const int kk = blockIdx.x;
  if (rs[kk].done) {
    if (threadIdx.x == 0) gate[kk].done = 1;
    return;
  }
  const cd* rk = r + (int64_t)kk * n;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += rk[i].re * rk[i].re + rk[i].im * rk[i].im;
  const double beta = sqrt(block_sum(s, red));
  cd* v0 = V + (int64_t)kk * (m + 1) * n;
  const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v0[i] = cscale(rk[i], inv);
  if (threadIdx.x == 0) {
    gs[kk].j = 0;
    gs[kk].beta = beta;
    gs[kk].resid = beta;
    gs[kk].target = 0.5 * tol * rs[kk].scale;
    g[(int64_t)kk * (m + 1)] = {beta, 0.0};
    gate[kk].done = beta > 0.0 ? 0 : 1;
  }
}

// w = A z with FP32 products and sums (z rounded to FP32 after scaling); warp per row.
__global__ void __launch_bounds__(512) k_gm_matvec(const cf* __restrict__ A, int n, int64_t ld, int64_t bstride,
                                                   const cd* __restrict__ Z, cd* __restrict__ V, int m, int j,
                                                   const RefineState* __restrict__ gate) {
  extern __shared__ float2 zs[];
  __shared__ double s_scale;
  const int kk = blockIdx.y;
  if (gate[kk].done) return;
  const cd* z = Z + ((int64_t)kk * m + j) * n;
  if (threadIdx.x == 0) s_scale = 0.0;
  __syncthreads();
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fmax(fabs(z[i].re), fabs(z[i].im)));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long*)&s_scale, __double_as_longlong(mx));
  __syncthreads();
  const double sc = s_scale > 0.0 ? s_scale : 1.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) zs[i] = make_float2((float)(z[i].re / sc), (float)(z[i].im / sc));
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 16 + warp;
  if (i >= n) return;
  const cf* row = A + (int64_t)kk * bstride + (int64_t)i * ld;
  float sr = 0.f, si = 0.f;
  for (int c = lane; c < n; c += 32) {
    const cf a = row[c];
    const float2 v = zs[c];
    sr = fmaf(a.re, v.x, fmaf(-a.im, v.y, sr));
    si = fmaf(a.re, v.y, fmaf(a.im, v.x, si));
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) V[((int64_t)kk * (m + 1) + j + 1) * n + i] = {(double)sr * sc, (double)si * sc};
}

// Arnoldi step j: orthogonalise w = V_{j+1} against V_0..V_j (classical Gram-Schmidt, twice),
// normalise, apply the previous Givens rotations to the new Hessenberg column, form the new
// rotation, update g, and close the cycle when |g_{j+1}| <= inner_tol * beta or j + 1 = m.
__global__ void __launch_bounds__(1024) k_gm_arnoldi(int n, int m, int j, cd* __restrict__ V, cd* __restrict__ H,
                                                     double* __restrict__ cs, cd* __restrict__ sn, cd* __restrict__ g,
                                                     GmresState* __restrict__ gs, RefineState* __restrict__ gate,
                                                     double inner_tol) {
  __shared__ double red[32];
  __shared__ cd hcol[64];   // m <= 62
  __shared__ cd hpass[64];
  const int kk = blockIdx.x;
  if (gate[kk].done) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  cd* Vk = V + (int64_t)kk * (m + 1) * n;
  cd* w = Vk + (int64_t)(j + 1) * n;
  if (tid <= j) hcol[tid] = {0.0, 0.0};
  for (int pass = 0; pass < 2; ++pass) {
    __syncthreads();
    // h_i = <v_i, w> for i = 0..j: warp per basis vector
    for (int i = warp; i <= j; i += nw) {
      const cd* vi = Vk + (int64_t)i * n;
      double sr = 0.0, si = 0.0;
      for (int t = lane; t < n; t += 32) {
        const cd a = vi[t], b = w[t];
        sr += a.re * b.re + a.im * b.im;  // conj(a) b
        si += a.re * b.im - a.im * b.re;
      }
      for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
      }
      if (lane == 0) hpass[i] = {sr, si};
    }
    __syncthreads();
    // w -= sum_i h_i v_i
    for (int t = tid; t < n; t += blockDim.x) {
      cd acc = w[t];
      for (int i = 0; i <= j; ++i) acc = csub(acc, cmul(hpass[i], Vk[(int64_t)i * n + t]));
      w[t] = acc;
    }
    if (tid <= j) hcol[tid] = cadd(hcol[tid], hpass[tid]);
  }
  __syncthreads();
  double s = 0.0;
  for (int t = tid; t < n; t += blockDim.x) s += w[t].re * w[t].re + w[t].im * w[t].im;
  const double hn = sqrt(block_sum(s, red));
  const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  for (int t = tid; t < n; t += blockDim.x) w[t] = cscale(w[t], inv);
  if (tid == 0) {
    cd* Hk = H + (int64_t)kk * (m + 1) * m;  // column-major: H[col * (m + 1) + row]
    double* ck = cs + (int64_t)kk * m;
    cd* sk = sn + (int64_t)kk * m;
    cd* gk = g + (int64_t)kk * (m + 1);
    cd col[64];
    for (int i = 0; i <= j; ++i) col[i] = hcol[i];
    col[j + 1] = {hn, 0.0};
    for (int i = 0; i < j; ++i) {  // previous rotations
      const cd a = col[i], b = col[i + 1];
      const cd sc = sk[i];
      col[i] = cadd(cscale(a, ck[i]), cmul(sc, b));
      col[i + 1] = csub(cscale(b, ck[i]), cmul(cd{sc.re, -sc.im}, a));
    }
    // new rotation zeroing col[j+1] (real, >= 0) under col[j]
    const cd a = col[j];
    const double b = col[j + 1].re, am = hypot(a.re, a.im), rr = hypot(am, b);
    double c;
    cd sv;
    if (am == 0.0) {
      c = 0.0;
      sv = {1.0, 0.0};
    } else {
      c = am / rr;
      sv = {a.re / am * b / rr, a.im / am * b / rr};
    }
    ck[j] = c;
    sk[j] = sv;
    col[j] = am == 0.0 ? cd{b, 0.0} : cd{a.re / am * rr, a.im / am * rr};
    col[j + 1] = {0.0, 0.0};
    for (int i = 0; i <= j + 1; ++i) Hk[(int64_t)j * (m + 1) + i] = col[i];
    const cd gj = gk[j];
    gk[j] = cscale(gj, c);
    gk[j + 1] = cscale(cmul(cd{-sv.re, sv.im}, gj), 1.0);  // -conj(s) g_j
    const double res = hypot(gk[j + 1].re, gk[j + 1].im);
    gs[kk].j = j + 1;
    gs[kk].iters += 1;
    gs[kk].resid = res;
    if (res <= fmax(inner_tol * gs[kk].beta, gs[kk].target) || j + 1 >= m || hn == 0.0) gate[kk].done = 1;
  }
}

// x += Z y with R y = g (R the rotated Hessenberg, j x j upper triangular).
__global__ void __launch_bounds__(1024) k_gm_update(int n, int m, const cd* __restrict__ Z, const cd* __restrict__ H,
                                                    const cd* __restrict__ g, const GmresState* __restrict__ gs,
                                                    const RefineState* __restrict__ rs, cd* __restrict__ x) {
  __shared__ cd y[64];
  const int kk = blockIdx.x;
  if (rs[kk].done) return;
  const int jn = gs[kk].j;
  if (jn <= 0) return;
  if (threadIdx.x == 0) {
    const cd* Hk = H + (int64_t)kk * (m + 1) * m;
    const cd* gk = g + (int64_t)kk * (m + 1);
    for (int i = jn - 1; i >= 0; --i) {
      cd s = gk[i];
      for (int c = i + 1; c < jn; ++c) s = csub(s, cmul(Hk[(int64_t)c * (m + 1) + i], y[c]));
      const cd d = Hk[(int64_t)i * (m + 1) + i];
      const double den = d.re * d.re + d.im * d.im;
      y[i] = den > 0.0 ? cd{(s.re * d.re + s.im * d.im) / den, (s.im * d.re - s.re * d.im) / den} : cd{0.0, 0.0};
    }
  }
  __syncthreads();
  const cd* Zk = Z + (int64_t)kk * m * n;
  cd* xk = x + (int64_t)kk * n;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    cd acc = xk[t];
    for (int i = 0; i < jn; ++i) acc = cadd(acc, cmul(y[i], Zk[(int64_t)i * n + t]));
    xk[t] = acc;
  }
}

__global__ void k_gm_collect(int nk, const GmresState* __restrict__ gs, RefineState* __restrict__ rs) {
  const int kk = blockIdx.x * blockDim.x + threadIdx.x;
  if (kk < nk) rs[kk].iters = gs[kk].iters;
}

size_t gmres_scratch_bytes(int nk, int n, int m) {
  auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
  return a((size_t)nk * (m + 1) * n * sizeof(cd)) + a((size_t)nk * m * n * sizeof(cd)) +
         a((size_t)nk * (m + 1) * m * sizeof(cd)) + a((size_t)nk * m * sizeof(double)) + a((size_t)nk * m * sizeof(cd)) +
         a((size_t)nk * (m + 1) * sizeof(cd)) + a((size_t)nk * sizeof(GmresState)) + a((size_t)nk * sizeof(RefineState)) +
         a((size_t)nk * n * sizeof(cd)) + a((size_t)nk * n * sizeof(double)) + 256;
}

// Solves A_kk x_kk = b_kk for kk < nk (A: FP32 systems with pitch ld, batch stride bstride),
// starting from x (in/out), preconditioned by factor sel[kk] of LU/perm (with the factors'
// diagonal-block inverses Dinv, or NULL).  state_dev receives a
// RefineState per system (done, iters = Arnoldi steps, backward error).
int gmres_solve(bie_ctx* c, const cf* A, int nk, int n, int64_t ld, int64_t bstride, const cd* b, cd* x,
                const cf* LU, int64_t lu_bstride, const int32_t* perm, const cf* Dinv, const int32_t* sel, int m,
                int cycles, double inner_tol, double tol, void* scratch, void* state_dev) {
  const int64_t dstride = diag_inv_stride(n);
  if (m < 1 || m > 62) return fail(BIE_ERR_INVALID_ARG, "gmres.m must be in [1, 62]");
  char* p = (char*)scratch;
  auto take = [&](size_t bytes) { char* q = p; p += (bytes + 255) & ~(size_t)255; return (void*)q; };
  cd* V = (cd*)take((size_t)nk * (m + 1) * n * sizeof(cd));
  cd* Z = (cd*)take((size_t)nk * m * n * sizeof(cd));
  cd* H = (cd*)take((size_t)nk * (m + 1) * m * sizeof(cd));
  double* cs = (double*)take((size_t)nk * m * sizeof(double));
  cd* sn = (cd*)take((size_t)nk * m * sizeof(cd));
  cd* g = (cd*)take((size_t)nk * (m + 1) * sizeof(cd));
  GmresState* gs = (GmresState*)take((size_t)nk * sizeof(GmresState));
  RefineState* gate = (RefineState*)take((size_t)nk * sizeof(RefineState));
  cd* r = (cd*)take((size_t)nk * n * sizeof(cd));
  double* rowabs = (double*)take((size_t)nk * n * sizeof(double));
  RefineState* rs = (RefineState*)state_dev;
  BIE_CUDA_TRY(cudaMemsetAsync(rs, 0, nk * sizeof(RefineState), c->stream));
  BIE_CUDA_TRY(cudaMemsetAsync(gs, 0, nk * sizeof(GmresState), c->stream));
  const size_t sm_trsv = (size_t)n * sizeof(cf), sm_mv = (size_t)n * sizeof(float2);
  if (sm_trsv > 200 * 1024) return fail(BIE_ERR_INVALID_ARG, "N too large for the shared-memory Krylov kernels");
  BIE_TRY((set_smem_max(k_trsv_lu)));
  BIE_TRY((set_smem_max(k_gm_matvec)));
  dim3 gr((unsigned)((n + 15) / 16), nk);
  for (int cy = 0; cy <= cycles; ++cy) {
    BIE_TRY(residual_ff(c, A, n, ld, bstride, nk, b, x, r, rowabs, rs));
    BIE_LAUNCH(k_refine_check<<<nk, 256, 0, c->stream>>>(n, b, x, r, rowabs, rs, tol, 0));
    if (cy == cycles) break;
    BIE_LAUNCH(k_gm_start<<<nk, 1024, 0, c->stream>>>(n, m, r, V, g, gs, rs, gate, tol));
    for (int j = 0; j < m; ++j) {
      // z_j = M^{-1} v_j
      BIE_LAUNCH(k_trsv_lu<<<nk, 1024, sm_trsv, c->stream>>>(LU, n, ld, lu_bstride, perm, V, Z, 0, gate, sel,
                                                             (int64_t)(m + 1) * n, (int64_t)j * n, (int64_t)m * n,
                                                             (int64_t)j * n, Dinv, dstride));
      BIE_LAUNCH(k_gm_matvec<<<gr, 512, sm_mv, c->stream>>>(A, n, ld, bstride, Z, V, m, j, gate));
      BIE_LAUNCH(k_gm_arnoldi<<<nk, 1024, 0, c->stream>>>(n, m, j, V, H, cs, sn, g, gs, gate, inner_tol));
    }
    BIE_LAUNCH(k_gm_update<<<nk, 1024, 0, c->stream>>>(n, m, Z, H, g, gs, rs, x));
  }
  BIE_LAUNCH(k_gm_collect<<<(nk + 127) / 128, 128, 0, c->stream>>>(nk, gs, rs));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

}  // namespace bie
