// refine.cu -- iterative refinement of the mixed-precision solves:
//   x_0 = (LU)^{-1} b;  repeat  r = b - A x  (A the FP32-assembled matrix, products and sums in
//   float-float, r in FP64);  stop when ||r||_inf <= tol (||A||_inf ||x||_inf + ||b||_inf);
//   d = (LU)^{-1} r (FP32);  x += d (FP64).
// Convergence is tracked per wavenumber on the device, so the host enqueues a fixed number of
// iterations without synchronising; kernels of converged systems return at once.
#include "bie_common.cuh"

namespace bie {


// ---- permutation vector from the LU's row interchanges: y = P r  <=>  y[i] = r[perm[i]] ----
__global__ void k_piv_to_perm(const int32_t* __restrict__ piv, int n, int32_t* __restrict__ perm) {
  extern __shared__ int32_t sp[];
  const int32_t* pv = piv + (int64_t)blockIdx.x * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sp[i] = i;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int s = 0; s < n; ++s) {
      int p = pv[s];
      int t = sp[s]; sp[s] = sp[p]; sp[p] = t;
    }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) perm[(int64_t)blockIdx.x * n + i] = sp[i];
}

// ---- triangular solves x = U^{-1} L^{-1} P r with one CTA (1024 threads) per system ---------
// The vector lives in shared memory; the factor is swept in 64-column blocks: the diagonal block
// is applied as a product with its precomputed inverse (all warps; k_diag_inv), or solved row by
// row by one warp when no inverse is given, then all warps update the remaining rows, eight rows
// per warp in flight.
constexpr int TB = 64;

// Inverses of the 64 x 64 diagonal blocks of L (unit lower) and U of every factor, by column-wise
// substitution in shared memory (thread j computes column j).  D: [nk][nblk][2][64][64] (L, U),
// rows and columns beyond the matrix are zero.  grid (nblk, nk, 2), block 64.
__global__ void __launch_bounds__(64) k_diag_inv(const cf* __restrict__ LU, int n, int64_t ld, int64_t bstride,
                                                 cf* __restrict__ D, int64_t dstride) {
  extern __shared__ cf smi[];
  cf* Ms = smi;            // [64][65]
  cf* X = smi + 64 * 65;   // [64][65]
  const int blk = blockIdx.x, kk = blockIdx.y, upper = blockIdx.z, j = threadIdx.x;
  const int j0 = blk * TB, bs = min(TB, n - j0);
  const cf* Mg = LU + (int64_t)kk * bstride + (int64_t)j0 * ld + j0;
  for (int idx = j; idx < TB * TB; idx += TB) {
    const int r = idx / TB, cc = idx % TB;
    Ms[r * 65 + cc] = (r < bs && cc < bs) ? Mg[(int64_t)r * ld + cc] : cf{0.f, 0.f};
  }
  __syncthreads();
  if (!upper) {
    for (int i = 0; i < TB; ++i) {
      float xr = (i == j) ? 1.f : 0.f, xi = 0.f;
      for (int m = j; m < i; ++m) {
        const cf a = Ms[i * 65 + m], b = X[m * 65 + j];
        xr -= a.re * b.re - a.im * b.im;
        xi -= a.re * b.im + a.im * b.re;
      }
      X[i * 65 + j] = (i < bs && j < bs) ? cf{xr, xi} : cf{0.f, 0.f};
    }
  } else {
    for (int i = TB - 1; i >= 0; --i) {
      float xr = (i == j) ? 1.f : 0.f, xi = 0.f;
      if (i < bs && j < bs) {
        for (int m = i + 1; m <= j; ++m) {
          const cf a = Ms[i * 65 + m], b = X[m * 65 + j];
          xr -= a.re * b.re - a.im * b.im;
          xi -= a.re * b.im + a.im * b.re;
        }
        const cf d = Ms[i * 65 + i];
        const float den = d.re * d.re + d.im * d.im;
        X[i * 65 + j] = {(xr * d.re + xi * d.im) / den, (xi * d.re - xr * d.im) / den};
      } else {
        X[i * 65 + j] = {0.f, 0.f};
      }
    }
  }
  __syncthreads();
  cf* Db = D + (int64_t)kk * dstride + ((int64_t)blk * 2 + upper) * TB * TB;
  for (int idx = j; idx < TB * TB; idx += TB) Db[idx] = X[(idx / TB) * 65 + idx % TB];
}

template <bool LOWER>
__device__ void trsv_sweep(const cf* __restrict__ M, int n, int64_t ld, cf* y, const cf* __restrict__ D, cf* ytmp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nblk = (n + TB - 1) / TB;
  for (int bi = 0; bi < nblk; ++bi) {
    const int blk = LOWER ? bi : nblk - 1 - bi;
    const int j0 = blk * TB, j1 = min(j0 + TB, n);
    if (D) {  // diagonal block: y_blk = inv(block) y_blk, one warp per row
      const cf* Db = D + ((int64_t)blk * 2 + (LOWER ? 0 : 1)) * TB * TB;
      const int bs = j1 - j0;
      for (int r = warp; r < bs; r += nw) {
        float sr = 0.f, si = 0.f;
        for (int cc = lane; cc < bs; cc += 32) {
          const cf d = Db[r * TB + cc];
          const cf v = y[j0 + cc];
          sr += d.re * v.re - d.im * v.im;
          si += d.re * v.im + d.im * v.re;
        }
        for (int o = 16; o > 0; o >>= 1) {
          sr += __shfl_xor_sync(0xffffffffu, sr, o);
          si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (lane == 0) ytmp[r] = {sr, si};
      }
      __syncthreads();
      if ((int)threadIdx.x < bs) y[j0 + threadIdx.x] = ytmp[threadIdx.x];
    } else if (warp == 0) {  // diagonal block, row by row
      for (int t = 0; t < j1 - j0; ++t) {
        const int r = LOWER ? j0 + t : j1 - 1 - t;
        float sr = 0.f, si = 0.f;
        for (int c = j0 + lane; c < j1; c += 32) {
          if (LOWER ? (c < r) : (c > r)) {
            const cf l = M[(int64_t)r * ld + c];
            const cf v = y[c];
            sr += l.re * v.re - l.im * v.im;
            si += l.re * v.im + l.im * v.re;
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          sr += __shfl_xor_sync(0xffffffffu, sr, o);
          si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (lane == 0) {
          cf v = {y[r].re - sr, y[r].im - si};
          if (!LOWER) {
            const cf d = M[(int64_t)r * ld + r];
            const float den = d.re * d.re + d.im * d.im;
            v = {(v.re * d.re + v.im * d.im) / den, (v.im * d.re - v.re * d.im) / den};
          }
          y[r] = v;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // update rows outside the block: lower -> rows >= j1, upper -> rows < j0
    const int rlo = LOWER ? j1 : 0, rhi = LOWER ? n : j0;
    const int c0 = j0 + 2 * lane;  // each lane holds two columns of the block
    cf ya = {0.f, 0.f}, yb = {0.f, 0.f};
    if (c0 < j1) ya = y[c0];
    if (c0 + 1 < j1) yb = y[c0 + 1];
    for (int r0 = rlo + warp * 8; r0 < rhi; r0 += nw * 8) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int r = r0 + u;
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < rhi) {
          const cf* p = M + (int64_t)r * ld + c0;
          if (c0 + 1 < j1) v[u] = *reinterpret_cast<const float4*>(p);
          else if (c0 < j1) v[u] = make_float4(p[0].re, p[0].im, 0.f, 0.f);
        }
      }
      // the 16 partial sums (8 rows x re, im) are reduced across the warp by halving exchanges:
      // at offset 16, 8, 4, 2 each lane keeps half of its values and adds its partner's copy of
      // them (8 + 4 + 2 + 1 shuffles), then one exchange at offset 1 completes the sums; lane L
      // ends with value 8 b4 + 4 b3 + 2 b2 + b1 (b_i the bits of L) = row (that >> 1), part (& 1)
      float t[16];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        t[2 * u] = v[u].x * ya.re - v[u].y * ya.im + v[u].z * yb.re - v[u].w * yb.im;
        t[2 * u + 1] = v[u].x * ya.im + v[u].y * ya.re + v[u].z * yb.im + v[u].w * yb.re;
      }
#pragma unroll
      for (int h = 8; h >= 1; h >>= 1) {
        const bool up = (lane & (2 * h)) != 0;
#pragma unroll
        for (int j = 0; j < h; ++j) {
          const float send = up ? t[j] : t[j + h];
          const float keep = up ? t[j + h] : t[j];
          t[j] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * h);
        }
      }
      t[0] += __shfl_xor_sync(0xffffffffu, t[0], 1);
      if ((lane & 1) == 0) {
        const int idx = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
        const int r = r0 + (idx >> 1);
        if (r < rhi) {
          if (idx & 1) y[r].im -= t[0];
          else y[r].re -= t[0];
        }
      }
    }
    __syncthreads();
  }
}

// rhs: cd vectors of n entries, system kk's at rhs + kk * rstride + roff (FP64); the solution is
// written to out + kk * ostride + ooff (added to it if accumulate).
// sel (optional): system blockIdx.x uses factor sel[blockIdx.x] (vectors stay indexed by blockIdx.x).
__global__ void __launch_bounds__(1024) k_trsv_lu(const cf* __restrict__ LU, int n, int64_t ld, int64_t bstride,
                                                  const int32_t* __restrict__ perm, const cd* __restrict__ rhs,
                                                  cd* __restrict__ out, int accumulate,
                                                  const RefineState* __restrict__ st,
                                                  const int32_t* __restrict__ sel, int64_t rstride, int64_t roff,
                                                  int64_t ostride, int64_t ooff, const cf* __restrict__ Dinv,
                                                  int64_t dstride) {
  extern __shared__ cf yv[];
  __shared__ cf ytmp[TB];
  const int kk = blockIdx.x;
  if (st && st[kk].done) return;
  const int fk = sel ? sel[kk] : kk;
  const cf* M = LU + (int64_t)fk * bstride;
  const int32_t* pm = perm + (int64_t)fk * n;
  const cd* r = rhs + (int64_t)kk * rstride + roff;
  // scale the right-hand side to O(1) before rounding it to FP32
  __shared__ double s_scale;
  if (threadIdx.x == 0) s_scale = 0.0;
  __syncthreads();
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fmax(fabs(r[i].re), fabs(r[i].im)));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long*)&s_scale, __double_as_longlong(mx));
  __syncthreads();
  const double sc = s_scale > 0.0 ? s_scale : 1.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const cd v = r[pm[i]];
    yv[i] = {(float)(v.re / sc), (float)(v.im / sc)};
  }
  __syncthreads();
  const cf* Df = Dinv ? Dinv + (int64_t)fk * dstride : nullptr;
  trsv_sweep<true>(M, n, ld, yv, Df, ytmp);
  trsv_sweep<false>(M, n, ld, yv, Df, ytmp);
  cd* o = out + (int64_t)kk * ostride + ooff;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const cd v = {(double)yv[i].re * sc, (double)yv[i].im * sc};
    o[i] = accumulate ? cadd(o[i], v) : v;
  }
}

// ---- the same solves for a few large systems: diagonal super-blocks and wide products ---------
// k_trsv_lu gives each system one CTA, whose bandwidth (about 180 GB/s) bounds a solve of a few
// large systems (9 systems of N = 20 544: 9 of 152 SMs busy).  Here the factor is taken in
// super-blocks of kSuper rows: one CTA per system solves the diagonal super-block (the blocked
// sweep of k_trsv_lu on that range, with the same diagonal-block inverses), then a launch over all
// SMs subtracts the super-block's columns times its solved entries from the rows outside it (below
// it for L, above it for U).  The solution lives in a global FP32 vector y (scaled to O(1) as in
// k_trsv_lu, the scale kept per system) between the launches.
constexpr int kSuper = 1024;
int64_t diag_inv_stride(int n);

// y = P rhs / scale (scale = max |rhs| component), one CTA per system
__global__ void __launch_bounds__(1024) k_trsv_begin(const int32_t* __restrict__ perm, const cd* __restrict__ rhs,
                                                     int n, const RefineState* __restrict__ st,
                                                     const int32_t* __restrict__ sel, cf* __restrict__ y,
                                                     double* __restrict__ scales) {
  const int kk = blockIdx.x;
  if (st && st[kk].done) return;
  const int fk = sel ? sel[kk] : kk;
  const int32_t* pm = perm + (int64_t)fk * n;
  const cd* r = rhs + (int64_t)kk * n;
  __shared__ double s_scale;
  if (threadIdx.x == 0) s_scale = 0.0;
  __syncthreads();
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fmax(fabs(r[i].re), fabs(r[i].im)));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long*)&s_scale, __double_as_longlong(mx));
  __syncthreads();
  const double sc = s_scale > 0.0 ? s_scale : 1.0;
  if (threadIdx.x == 0) scales[kk] = sc;
  cf* yk = y + (int64_t)kk * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const cd v = r[pm[i]];
    yk[i] = {(float)(v.re / sc), (float)(v.im / sc)};
  }
}

// diagonal super-block [s0, s1) of system kk's L (LOWER) or U, in place on y; one CTA per system
template <bool LOWER>
__global__ void __launch_bounds__(1024) k_trsv_super(const cf* __restrict__ LU, int n, int64_t ld, int64_t bstride,
                                                     const RefineState* __restrict__ st,
                                                     const int32_t* __restrict__ sel, cf* __restrict__ y, int s0,
                                                     int s1, const cf* __restrict__ Dinv, int64_t dstride) {
  __shared__ cf ys[kSuper];
  __shared__ cf ytmp[TB];
  const int kk = blockIdx.x;
  if (st && st[kk].done) return;
  const int fk = sel ? sel[kk] : kk;
  const cf* M = LU + (int64_t)fk * bstride + (int64_t)s0 * ld + s0;
  cf* yk = y + (int64_t)kk * n;
  const int m = s1 - s0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) ys[i] = yk[s0 + i];
  __syncthreads();
  const cf* Df = Dinv ? Dinv + (int64_t)fk * dstride + (int64_t)(s0 / TB) * 2 * TB * TB : nullptr;
  trsv_sweep<LOWER>(M, m, ld, ys, Df, ytmp);
  for (int i = threadIdx.x; i < m; i += blockDim.x) yk[s0 + i] = ys[i];
}

// rows [r0, r1) of system kk: y[r] -= sum over c in [s0, s1) of F[r][c] y[c]; a warp takes 8 rows,
// the super-block's entries of y are staged in shared memory.  grid (ceil((r1 - r0) / 64), nk),
// block 256.
__global__ void __launch_bounds__(256) k_trsv_gemv(const cf* __restrict__ LU, int n, int64_t ld, int64_t bstride,
                                                   const RefineState* __restrict__ st,
                                                   const int32_t* __restrict__ sel, cf* __restrict__ y, int s0, int s1,
                                                   int r0, int r1) {
  constexpr int R = 8;
  __shared__ cf ys[kSuper];
  const int kk = blockIdx.y;
  if (st && st[kk].done) return;
  const int fk = sel ? sel[kk] : kk;
  cf* yk = y + (int64_t)kk * n;
  const int m = s1 - s0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) ys[i] = yk[s0 + i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = r0 + blockIdx.x * 64 + warp * R;
  if (i0 >= r1) return;
  const int nr = min(R, r1 - i0);
  const cf* F = LU + (int64_t)fk * bstride + (int64_t)i0 * ld + s0;
  float ar[R], ai[R];
#pragma unroll
  for (int u = 0; u < R; ++u) ar[u] = ai[u] = 0.f;
#pragma unroll 2
  for (int cc = lane; cc < m; cc += 32) {
    const cf v = ys[cc];
#pragma unroll
    for (int u = 0; u < R; ++u) {
      if (u < nr) {
        const cf f = F[(int64_t)u * ld + cc];
        ar[u] += f.re * v.re - f.im * v.im;
        ai[u] += f.re * v.im + f.im * v.re;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < R; ++u) {
    if (u >= nr) break;
    float a = ar[u], b = ai[u];
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      cf& t = yk[i0 + u];
      t.re -= a;
      t.im -= b;
    }
  }
}

// out (+)= y * scale
__global__ void k_trsv_end(const cf* __restrict__ y, const double* __restrict__ scales, int n,
                           const RefineState* __restrict__ st, cd* __restrict__ out, int accumulate) {
  const int kk = blockIdx.y;
  if (st && st[kk].done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double sc = scales[kk];
  const cf v = y[(int64_t)kk * n + i];
  cd& o = out[(int64_t)kk * n + i];
  const cd w = {(double)v.re * sc, (double)v.im * sc};
  o = accumulate ? cadd(o, w) : w;
}

size_t trsv_scratch_bytes(int nk, int n) { return 256 + (size_t)nk * n * sizeof(cf) + (size_t)nk * sizeof(double); }

// x (+)= (LU)^{-1} P rhs for nk systems (vectors [nk][n]; factor sel[kk] if sel); systems whose
// state is done are skipped.  The super-block form when the systems are few and large and
// `scratch` (trsv_scratch_bytes) is given, otherwise k_trsv_lu.
int trsv_solve(bie_ctx* c, const cf* LU, int nk, int n, int64_t ld, int64_t bstride, const int32_t* perm,
               const cd* rhs, cd* out, int accumulate, const RefineState* st, const int32_t* sel, const cf* D,
               void* scratch) {
  const int64_t dstride = diag_inv_stride(n);
  int nsm = 0;
  BIE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
  if (!scratch || !D || n < 4 * kSuper || 2 * nk > nsm) {
    BIE_TRY((set_smem_max(k_trsv_lu)));
    BIE_LAUNCH(k_trsv_lu<<<nk, 1024, (size_t)n * sizeof(cf), c->stream>>>(LU, n, ld, bstride, perm, rhs, out, accumulate,
                                                                        st, sel, n, 0, n, 0, D, dstride));
    return BIE_OK;
  }
  double* scales = (double*)scratch;
  cf* y = (cf*)((char*)scratch + (((size_t)nk * sizeof(double) + 255) & ~(size_t)255));
  BIE_LAUNCH(k_trsv_begin<<<nk, 1024, 0, c->stream>>>(perm, rhs, n, st, sel, y, scales));
  const int ns = (n + kSuper - 1) / kSuper;
  for (int b = 0; b < ns; ++b) {  // L: super-blocks in order, then the rows below
    const int s0 = b * kSuper, s1 = std::min(n, s0 + kSuper);
    BIE_LAUNCH(k_trsv_super<true><<<nk, 1024, 0, c->stream>>>(LU, n, ld, bstride, st, sel, y, s0, s1, D, dstride));
    if (s1 < n) {
      dim3 g((unsigned)((n - s1 + 63) / 64), nk);
      BIE_LAUNCH(k_trsv_gemv<<<g, 256, 0, c->stream>>>(LU, n, ld, bstride, st, sel, y, s0, s1, s1, n));
    }
  }
  for (int b = ns - 1; b >= 0; --b) {  // U: super-blocks in reverse, then the rows above
    const int s0 = b * kSuper, s1 = std::min(n, s0 + kSuper);
    BIE_LAUNCH(k_trsv_super<false><<<nk, 1024, 0, c->stream>>>(LU, n, ld, bstride, st, sel, y, s0, s1, D, dstride));
    if (s0 > 0) {
      dim3 g((unsigned)((s0 + 63) / 64), nk);
      BIE_LAUNCH(k_trsv_gemv<<<g, 256, 0, c->stream>>>(LU, n, ld, bstride, st, sel, y, s0, s1, 0, s0));
    }
  }
  dim3 ge((unsigned)((n + 255) / 256), nk);
  BIE_LAUNCH(k_trsv_end<<<ge, 256, 0, c->stream>>>(y, scales, n, st, out, accumulate));
  return BIE_OK;
}

// ---- residual r = b - A x in float-float; also the row sums of |A| for ||A||_inf ------------
// grid (ceil(n / 16), batch), block 512: one warp per row, x staged in shared memory as ff.
__device__ __forceinline__ void ff_acc_prod(float a, float xh, float xl, float& sh, float& sl) {
  const float p = a * xh;
  float e = __fmaf_rn(a, xh, -p);
  e = __fmaf_rn(a, xl, e);
  const ff t = ff_two_sum(sh, p);
  sh = t.hi;
  sl += t.lo + e;
}

// stage: x split into float-float once per CTA in shared memory (n * 16 bytes); otherwise (large n)
// every lane splits the FP64 entries it reads.
__global__ void __launch_bounds__(512) k_residual_ff(const cf* __restrict__ A, int n, int64_t ld, int64_t bstride,
                                                     const cd* __restrict__ b, const cd* __restrict__ x,
                                                     cd* __restrict__ r, double* __restrict__ rowabs,
                                                     const RefineState* __restrict__ st, int stage) {
  extern __shared__ float4 xs[];  // [n]: re_hi, re_lo, im_hi, im_lo
  const int kk = blockIdx.y;
  if (st[kk].done) return;
  const cd* xk = x + (int64_t)kk * n;
  if (stage) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const ff a = ff_from_double(xk[j].re), c = ff_from_double(xk[j].im);
      xs[j] = make_float4(a.hi, a.lo, c.hi, c.lo);
    }
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 16 + warp;
  if (i >= n) return;
  const cf* row = A + (int64_t)kk * bstride + (int64_t)i * ld;
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f, ab = 0.f;
  for (int j = lane; j < n; j += 32) {
    const cf a = row[j];
    float4 v;
    if (stage) {
      v = xs[j];
    } else {
      const ff p = ff_from_double(xk[j].re), q = ff_from_double(xk[j].im);
      v = make_float4(p.hi, p.lo, q.hi, q.lo);
    }
    ff_acc_prod(a.re, v.x, v.y, rh, rl);
    ff_acc_prod(-a.im, v.z, v.w, rh, rl);
    ff_acc_prod(a.re, v.z, v.w, ih, il);
    ff_acc_prod(a.im, v.x, v.y, ih, il);
    ab += fabsf(a.re) + fabsf(a.im);
  }
  double sr = (double)rh + (double)rl, si = (double)ih + (double)il, sa = ab;
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
  }
  if (lane == 0) {
    const cd bi = b[(int64_t)kk * n + i];
    r[(int64_t)kk * n + i] = {bi.re - sr, bi.im - si};
    rowabs[(int64_t)kk * n + i] = sa;
  }
}

// The same residual for large n (x does not fit shared memory with several CTAs per SM): a warp
// takes 8 rows, so that each FP64 entry of x it reads is split into float-float once for 8 rows
// (the FP64 conversions of the one-row-per-warp form bounded it on the narrow FP64 pipe).
// grid (ceil(n / 64), batch), block 256.
__global__ void __launch_bounds__(256) k_residual_ff_r8(const cf* __restrict__ A, int n, int64_t ld, int64_t bstride,
                                                        const cd* __restrict__ b, const cd* __restrict__ x,
                                                        cd* __restrict__ r, double* __restrict__ rowabs,
                                                        const RefineState* __restrict__ st) {
  constexpr int R = 8;
  const int kk = blockIdx.y;
  if (st[kk].done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = blockIdx.x * 64 + warp * R;
  if (i0 >= n) return;
  const int nr = min(R, n - i0);
  const cf* A0 = A + (int64_t)kk * bstride + (int64_t)i0 * ld;
  const cd* xk = x + (int64_t)kk * n;
  float rh[R], rl[R], ih[R], il[R], ab[R];
#pragma unroll
  for (int u = 0; u < R; ++u) rh[u] = rl[u] = ih[u] = il[u] = ab[u] = 0.f;
#pragma unroll 2
  for (int j = lane; j < n; j += 32) {
    const ff p = ff_from_double(xk[j].re), q = ff_from_double(xk[j].im);
#pragma unroll
    for (int u = 0; u < R; ++u) {
      if (u < nr) {
        const cf a = A0[(int64_t)u * ld + j];
        ff_acc_prod(a.re, p.hi, p.lo, rh[u], rl[u]);
        ff_acc_prod(-a.im, q.hi, q.lo, rh[u], rl[u]);
        ff_acc_prod(a.re, q.hi, q.lo, ih[u], il[u]);
        ff_acc_prod(a.im, p.hi, p.lo, ih[u], il[u]);
        ab[u] += fabsf(a.re) + fabsf(a.im);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < R; ++u) {
    if (u >= nr) break;
    double sr = (double)rh[u] + (double)rl[u], si = (double)ih[u] + (double)il[u], sa = ab[u];
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
    }
    if (lane == 0) {
      const int64_t t = (int64_t)kk * n + i0 + u;
      const cd bi = b[t];
      r[t] = {bi.re - sr, bi.im - si};
      rowabs[t] = sa;
    }
  }
}

// The residual of nk systems: x staged in shared memory while it fits four CTAs per SM,
// otherwise 8 rows per warp.
int residual_ff(bie_ctx* c, const cf* A, int n, int64_t ld, int64_t bstride, int nk, const cd* b, const cd* x, cd* r,
                double* rowabs, const RefineState* st) {
  if ((size_t)n * sizeof(float4) <= 48 * 1024) {
    BIE_TRY((set_smem_max(k_residual_ff)));
    dim3 gr((unsigned)((n + 15) / 16), nk);
    BIE_LAUNCH(k_residual_ff<<<gr, 512, (size_t)n * sizeof(float4), c->stream>>>(A, n, ld, bstride, b, x, r, rowabs, st, 1));
  } else {
    dim3 gr((unsigned)((n + 63) / 64), nk);
    BIE_LAUNCH(k_residual_ff_r8<<<gr, 256, 0, c->stream>>>(A, n, ld, bstride, b, x, r, rowabs, st));
  }
  return BIE_OK;
}

// ---- convergence test per system (one CTA each) ----------------------------------------------
__global__ void k_refine_check(int n, const cd* __restrict__ b, const cd* __restrict__ x, const cd* __restrict__ r,
                               const double* __restrict__ rowabs, RefineState* __restrict__ st, double tol,
                               int count_iter) {
  const int kk = blockIdx.x;
  if (st[kk].done) return;
  __shared__ double red[4][32];
  double rm = 0, xm = 0, bm = 0, am = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t t = (int64_t)kk * n + i;
    rm = fmax(rm, fmax(fabs(r[t].re), fabs(r[t].im)));
    xm = fmax(xm, fmax(fabs(x[t].re), fabs(x[t].im)));
    bm = fmax(bm, fmax(fabs(b[t].re), fabs(b[t].im)));
    am = fmax(am, rowabs[t]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    rm = fmax(rm, __shfl_xor_sync(0xffffffffu, rm, o));
    xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, o));
    bm = fmax(bm, __shfl_xor_sync(0xffffffffu, bm, o));
    am = fmax(am, __shfl_xor_sync(0xffffffffu, am, o));
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[0][w] = rm; red[1][w] = xm; red[2][w] = bm; red[3][w] = am; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int t = 1; t < (int)(blockDim.x >> 5); ++t) {
      rm = fmax(rm, red[0][t]); xm = fmax(xm, red[1][t]); bm = fmax(bm, red[2][t]); am = fmax(am, red[3][t]);
    }
    // b = 0 (a sound-hard body at k = 0) is solved exactly by x = 0: backward error 0, not 0/0
    const double den = am * xm + bm;
    const double be = den > 0.0 ? rm / den : (rm > 0.0 ? INFINITY : 0.0);
    st[kk].anorm = am;
    st[kk].bnorm = bm;
    st[kk].berr = be;
    st[kk].scale = am * xm + bm;
    if (be <= tol) st[kk].done = 1;
    else if (count_iter) st[kk].iters += 1;
  }
}

// ---- sensitivity of the solution to the FP32 assembly -----------------------------------------
// v = E x with E_ij = eps |A_ij| eta_ij, eta_ij a hashed unit value in {1, i, -1, -i}: a random
// perturbation of the size of the assembly's rounding.  z = (LU)^{-1} v then estimates the
// solution's error against the FP64-assembled system; near an interior resonance (Sec. 4's remark
// on w = 20.1a) ||z|| / ||x|| grows with the condition number and the system is re-solved in FP64.
// stage: x rounded to FP32 once per CTA into shared memory (n * 8 bytes); otherwise every lane
// rounds the FP64 entries it reads.  The magnitude |A_ij| comes from the FP32 reciprocal square
// root (a relative error of a few 1e-8 in a random perturbation's size).
__global__ void __launch_bounds__(512) k_perturb(const cf* __restrict__ A, int n, int64_t ld, int64_t bstride,
                                                 const cd* __restrict__ x, cd* __restrict__ v, float eps, int stage) {
  extern __shared__ float2 xs32[];  // [n]
  const int kk = blockIdx.y;
  const cd* xk = x + (int64_t)kk * n;
  if (stage) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) xs32[j] = make_float2((float)xk[j].re, (float)xk[j].im);
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 16 + warp;
  if (i >= n) return;
  const cf* row = A + (int64_t)kk * bstride + (int64_t)i * ld;
  float sr = 0.f, si = 0.f;
  for (int j = lane; j < n; j += 32) {
    const cf a = row[j];
    const float a2 = a.re * a.re + a.im * a.im;
    const float m = a2 > 0.f ? eps * (a2 * rsqrtf(a2)) : 0.f;
    uint32_t h = (uint32_t)i * 0x9E3779B1u ^ ((uint32_t)j * 0x85EBCA77u + 0x27D4EB2Fu);
    h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12;
    const uint32_t q = (h >> 30) & 3u;
    const float er = (q == 0) ? m : (q == 2 ? -m : 0.f), ei = (q == 1) ? m : (q == 3 ? -m : 0.f);
    const float2 xv = stage ? xs32[j] : make_float2((float)xk[j].re, (float)xk[j].im);
    sr += er * xv.x - ei * xv.y;
    si += er * xv.y + ei * xv.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) v[(int64_t)kk * n + i] = {(double)sr, (double)si};
}

// The same perturbation for large n: a warp takes 8 rows and rounds each entry of x it reads
// once for all of them (no shared-memory copy of x, which at large n left one CTA per SM).
// grid (ceil(n / 64), batch), block 256.
__global__ void __launch_bounds__(256) k_perturb_r8(const cf* __restrict__ A, int n, int64_t ld, int64_t bstride,
                                                    const cd* __restrict__ x, cd* __restrict__ v, float eps) {
  constexpr int R = 8;
  const int kk = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = blockIdx.x * 64 + warp * R;
  if (i0 >= n) return;
  const int nr = min(R, n - i0);
  const cf* A0 = A + (int64_t)kk * bstride + (int64_t)i0 * ld;
  const cd* xk = x + (int64_t)kk * n;
  float sr[R], si[R];
#pragma unroll
  for (int u = 0; u < R; ++u) sr[u] = si[u] = 0.f;
#pragma unroll 2
  for (int j = lane; j < n; j += 32) {
    const float2 xv = make_float2((float)xk[j].re, (float)xk[j].im);
#pragma unroll
    for (int u = 0; u < R; ++u) {
      if (u < nr) {
        const int i = i0 + u;
        const cf a = A0[(int64_t)u * ld + j];
        const float a2 = a.re * a.re + a.im * a.im;
        const float m = a2 > 0.f ? eps * (a2 * rsqrtf(a2)) : 0.f;
        uint32_t h = (uint32_t)i * 0x9E3779B1u ^ ((uint32_t)j * 0x85EBCA77u + 0x27D4EB2Fu);
        h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12;
        const uint32_t q = (h >> 30) & 3u;
        const float er = (q == 0) ? m : (q == 2 ? -m : 0.f), ei = (q == 1) ? m : (q == 3 ? -m : 0.f);
        sr[u] += er * xv.x - ei * xv.y;
        si[u] += er * xv.y + ei * xv.x;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < R; ++u) {
    if (u >= nr) break;
    float a = sr[u], b2 = si[u];
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b2 += __shfl_xor_sync(0xffffffffu, b2, o);
    }
    if (lane == 0) v[(int64_t)kk * n + i0 + u] = {(double)a, (double)b2};
  }
}

// The perturbation product of nk systems (x rounded once per CTA into shared memory while it
// fits four CTAs per SM, otherwise 8 rows per warp).
int perturb(bie_ctx* c, const cf* A, int n, int64_t ld, int64_t bstride, int nk, const cd* x, cd* v, float eps) {
  if ((size_t)n * sizeof(float2) <= 48 * 1024) {
    BIE_TRY((set_smem_max(k_perturb)));
    dim3 gr((unsigned)((n + 15) / 16), nk);
    BIE_LAUNCH(k_perturb<<<gr, 512, (size_t)n * sizeof(float2), c->stream>>>(A, n, ld, bstride, x, v, eps, 1));
  } else {
    dim3 gr((unsigned)((n + 63) / 64), nk);
    BIE_LAUNCH(k_perturb_r8<<<gr, 256, 0, c->stream>>>(A, n, ld, bstride, x, v, eps));
  }
  return BIE_OK;
}

__global__ void k_err_est(int n, const cd* __restrict__ x, const cd* __restrict__ z, RefineState* __restrict__ st) {
  const int kk = blockIdx.x;
  __shared__ double red[2][32];
  double zs = 0, xs = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t t = (int64_t)kk * n + i;
    zs += z[t].re * z[t].re + z[t].im * z[t].im;
    xs += x[t].re * x[t].re + x[t].im * x[t].im;
  }
  for (int o = 16; o > 0; o >>= 1) {
    zs += __shfl_xor_sync(0xffffffffu, zs, o);
    xs += __shfl_xor_sync(0xffffffffu, xs, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[0][w] = zs; red[1][w] = xs; }
  __syncthreads();
  if (threadIdx.x == 0) {
    zs = 0; xs = 0;
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) { zs += red[0][t]; xs += red[1][t]; }
    st[kk].err_est = xs > 0 ? sqrt(zs / xs) : 0.0;
  }
}

int64_t diag_inv_stride(int n) { return (int64_t)((n + TB - 1) / TB) * 2 * TB * TB; }

// Inverses of the diagonal blocks of nk factors (D: [nk][diag_inv_stride(n)] cf).
int diag_inverses(bie_ctx* c, const cf* LU, int nk, int n, int64_t ld, int64_t bstride, cf* D) {
  BIE_TRY((set_smem_max(k_diag_inv)));
  dim3 g((unsigned)((n + TB - 1) / TB), (unsigned)nk, 2);
  BIE_LAUNCH(k_diag_inv<<<g, TB, 2 * 64 * 65 * sizeof(cf), c->stream>>>(LU, n, ld, bstride, D, diag_inv_stride(n)));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

// The row permutations and diagonal-block inverses of nk factors (what refine_solve forms before
// its solves), for factors refined by refine_fp64_system directly.
int factor_aux(bie_ctx* c, const cf* LU, int nk, int n, int64_t ld, int64_t bstride, const int32_t* piv,
               int32_t* perm, cf* D) {
  if ((size_t)n * sizeof(int32_t) > 200 * 1024) return fail(BIE_ERR_INVALID_ARG, "N too large for the permutation kernel");
  BIE_TRY((set_smem_max(k_piv_to_perm)));
  BIE_LAUNCH(k_piv_to_perm<<<nk, 256, n * sizeof(int32_t), c->stream>>>(piv, n, perm));
  return diag_inverses(c, LU, nk, n, ld, bstride, D);
}

int refine_solve(bie_ctx* c, const cf* A, const cf* LU, int nk, int n, int64_t ld, int64_t bstride,
                 const int32_t* piv, const cd* b, cd* x, cd* r, double* rowabs, int32_t* perm, void* state_dev,
                 int it_max, double tol, cf* D, void* tscratch) {
  RefineState* st = (RefineState*)state_dev;
  BIE_CUDA_TRY(cudaMemsetAsync(st, 0, nk * sizeof(RefineState), c->stream));
  if ((size_t)n * sizeof(int32_t) > 200 * 1024) return fail(BIE_ERR_INVALID_ARG, "N too large for the permutation kernel");
  BIE_TRY((set_smem_max(k_piv_to_perm)));
  BIE_LAUNCH(k_piv_to_perm<<<nk, 256, n * sizeof(int32_t), c->stream>>>(piv, n, perm));
  if (D) BIE_TRY(diag_inverses(c, LU, nk, n, ld, bstride, D));
  const size_t sm_trsv = (size_t)n * sizeof(cf);
  if (sm_trsv > 200 * 1024)
    return fail(BIE_ERR_INVALID_ARG, "N too large for the shared-memory triangular solves (N <= 25600)");
  BIE_TRY(trsv_solve(c, LU, nk, n, ld, bstride, perm, b, x, 0, nullptr, nullptr, D, tscratch));
  for (int it = 0; it <= it_max; ++it) {
    BIE_TRY(residual_ff(c, A, n, ld, bstride, nk, b, x, r, rowabs, st));
    BIE_LAUNCH(k_refine_check<<<nk, 256, 0, c->stream>>>(n, b, x, r, rowabs, st, tol, it < it_max));
    if (it == it_max) break;
    BIE_TRY(trsv_solve(c, LU, nk, n, ld, bstride, perm, r, x, 1, st, nullptr, D, tscratch));
  }
  // assembly-sensitivity estimate (r is free now)
  BIE_TRY(perturb(c, A, n, ld, bstride, nk, x, r, 6e-8f));
  BIE_TRY(trsv_solve(c, LU, nk, n, ld, bstride, perm, r, r, 0, nullptr, nullptr, D, tscratch));
  BIE_LAUNCH(k_err_est<<<nk, 256, 0, c->stream>>>(n, x, r, st));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

size_t refine_state_bytes(int nk) { return (size_t)nk * sizeof(RefineState); }

// Right-hand sides b = -B known of nk systems from their known-column matrices B (the FP32
// entries multiplied exactly and summed in float-float, as the residual).  zero: scratch
// [nk][n], overwritten with zeros; rowabs, state: scratch.
int rhs_from_known(bie_ctx* c, const cf* B, int nk, int n, int64_t ld, int64_t bstride, const cd* known, cd* zero,
                   cd* b, double* rowabs, void* state_dev) {
  RefineState* st = (RefineState*)state_dev;
  BIE_CUDA_TRY(cudaMemsetAsync(st, 0, nk * sizeof(RefineState), c->stream));
  BIE_CUDA_TRY(cudaMemsetAsync(zero, 0, (size_t)nk * n * sizeof(cd), c->stream));
  BIE_TRY(residual_ff(c, B, n, ld, bstride, nk, zero, known, b, rowabs, st));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

// ---- refinement against the FP64-assembled system (wavenumbers flagged by the estimate) ------
// r = b64 - A64 x in FP64; corrections still come from the low-precision factor of the FP32
// system, which remains a good preconditioner while cond(A) * (its error) < 1.
__global__ void __launch_bounds__(512) k_residual64(const cd* __restrict__ A, int n, const cd* __restrict__ b,
                                                    const cd* __restrict__ x, cd* __restrict__ r,
                                                    double* __restrict__ rowabs, const RefineState* __restrict__ st) {
  const int g = blockIdx.y;
  if (st[g].done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 16 + warp;
  if (i >= n) return;
  const cd* row = A + ((int64_t)g * n + i) * n;
  const cd* xg = x + (int64_t)g * n;
  double sr = 0, si = 0, sa = 0;
  for (int j = lane; j < n; j += 32) {
    const cd a = row[j], v = xg[j];
    sr = fma(a.re, v.re, fma(-a.im, v.im, sr));
    si = fma(a.re, v.im, fma(a.im, v.re, si));
    sa += fabs(a.re) + fabs(a.im);
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
  }
  if (lane == 0) {
    const cd bi = b[(int64_t)g * n + i];
    r[(int64_t)g * n + i] = {bi.re - sr, bi.im - si};
    rowabs[(int64_t)g * n + i] = sa;
  }
}

// FP64 variant: B [nk][n][n] (cd), b = -B known with FP64 products and sums.
int rhs_from_known64(bie_ctx* c, const cd* B, int nk, int n, const cd* known, cd* zero, cd* b, double* rowabs,
                     void* state_dev) {
  RefineState* st = (RefineState*)state_dev;
  BIE_CUDA_TRY(cudaMemsetAsync(st, 0, nk * sizeof(RefineState), c->stream));
  BIE_CUDA_TRY(cudaMemsetAsync(zero, 0, (size_t)nk * n * sizeof(cd), c->stream));
  dim3 gr((unsigned)((n + 15) / 16), nk);
  BIE_LAUNCH(k_residual64<<<gr, 512, 0, c->stream>>>(B, n, zero, known, b, rowabs, st));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

__global__ void k_gather_scatter(cd* __restrict__ xb, cd* __restrict__ xg, const int32_t* __restrict__ sel, int n,
                                 int to_group) {
  const int g = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || sel[g] < 0) return;
  cd* src = to_group ? xb + (int64_t)sel[g] * n : xg + (int64_t)g * n;
  cd* dst = to_group ? xg + (int64_t)g * n : xb + (int64_t)sel[g] * n;
  dst[i] = src[i];
}

// Refines x[sel[g]] (g < ng) against A64/b64 [ng] with factors LU[sel[g]].  Scratch: xg, r [ng][n],
// rowabs [ng][n], state [ng] (zeroed here with reset_state; otherwise the caller's: a slot whose
// state is done, or whose selection is negative, is left alone).
int refine_fp64_system(bie_ctx* c, const cd* A64, const cd* b64, const cf* LU, int64_t ld, int64_t bstride,
                       const int32_t* perm, const int32_t* sel_dev, int ng, int n, cd* x, cd* xg, cd* r,
                       double* rowabs, void* state_dev, int it_max, double tol, const cf* D, void* tscratch,
                       bool reset_state) {
  RefineState* st = (RefineState*)state_dev;
  if (reset_state) BIE_CUDA_TRY(cudaMemsetAsync(st, 0, ng * sizeof(RefineState), c->stream));
  dim3 gv((unsigned)((n + 255) / 256), ng);
  BIE_LAUNCH(k_gather_scatter<<<gv, 256, 0, c->stream>>>(x, xg, sel_dev, n, 1));
  dim3 gr((unsigned)((n + 15) / 16), ng);
  for (int it = 0; it <= it_max; ++it) {
    BIE_LAUNCH(k_residual64<<<gr, 512, 0, c->stream>>>(A64, n, b64, xg, r, rowabs, st));
    BIE_LAUNCH(k_refine_check<<<ng, 256, 0, c->stream>>>(n, b64, xg, r, rowabs, st, tol, it < it_max));
    if (it == it_max) break;
    BIE_TRY(trsv_solve(c, LU, ng, n, ld, bstride, perm, r, xg, 1, st, sel_dev, D, tscratch));
  }
  BIE_LAUNCH(k_gather_scatter<<<gv, 256, 0, c->stream>>>(x, xg, sel_dev, n, 0));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int refine_read_state(bie_ctx* c, const void* state_dev, int nk, int32_t* done, int32_t* iters, double* berr,
                      double* err_est) {
  std::vector<RefineState> h(nk);
  BIE_CUDA_TRY(cudaMemcpyAsync(h.data(), state_dev, nk * sizeof(RefineState), cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < nk; ++i) {
    done[i] = h[i].done;
    iters[i] = h[i].iters;
    berr[i] = h[i].berr;
    err_est[i] = h[i].err_est;
  }
  return BIE_OK;
}

}  // namespace bie
