// field.cu -- scattered field at observation points by the boundary-regularised representation
// Eq. (BRIEFdmn) (Sec. 3).  With the S_inf integrals evaluated analytically (App. B reasoning,
// applied to g and f about the foot point x0 and to the source points x_p and x0):
//   4 pi P(x_p) = 4 pi P0 + int_S { Pt [dG(x_p,x) - dG(x0,x)] - [G(x_p,x) - G(x0,x)] dPt } dS,
//   Pt = P(x) - P0 g(x) - P0' f(x),  dPt = P'(x) - P0 dg(x) - P0' df(x),
// g = cos(k nu0.(x - x0)), f = sin(k nu0.(x - x0)) / k, x0 the closest surface point of x_p,
// nu0 the surface normal there, P0 and P0' interpolated quadratically at x0.
//
// Layout: the surface values are first interpolated to every standard quadrature point
// (k_interp_q), then each CTA owns a tile of observation points for one k and sweeps all
// quadrature points through shared memory (an N-body style tile loop).
#include "bie_common.cuh"

namespace bie {

// Pq[kk][p], Pnq[kk][p] = sum_a N_a(q) {P, P'}[node a of e], p = e*Q + q.
__global__ void k_interp_q64(const int32_t* __restrict__ elems, int64_t N, int64_t E, int Q,
                             const double* __restrict__ qshape, const cd* __restrict__ surf, cd* __restrict__ Pq,
                             cd* __restrict__ Pnq) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int kk = blockIdx.y;
  if (p >= E * Q) return;
  int64_t e = p / Q;
  int q = (int)(p % Q);
  const cd* P = surf + (int64_t)kk * 2 * N;
  const cd* Pn = P + N;
  cd a = {0, 0}, b = {0, 0};
  for (int t = 0; t < 6; ++t) {
    int32_t j = elems[6 * e + t];
    double s = qshape[q * 6 + t];
    a.re += s * P[j].re; a.im += s * P[j].im;
    b.re += s * Pn[j].re; b.im += s * Pn[j].im;
  }
  Pq[(int64_t)kk * E * Q + p] = a;
  Pnq[(int64_t)kk * E * Q + p] = b;
}

constexpr int FT = 128;  // points per CTA and quadrature points per shared tile

__global__ void __launch_bounds__(FT) k_field64(const int32_t* __restrict__ elems, int64_t N, int64_t EQ,
                                                const double* __restrict__ qgeo, const cd* __restrict__ Pq,
                                                const cd* __restrict__ Pnq, const cd* __restrict__ surf,
                                                const double* __restrict__ xp, int64_t M,
                                                const int32_t* __restrict__ foot_elem, const double* __restrict__ foot,
                                                const double* __restrict__ kv, cd* __restrict__ T) {
  __shared__ double sx[FT], sy[FT], sz[FT], snx[FT], sny[FT], snz[FT], sw[FT];
  __shared__ cd sP[FT], sPn[FT];
  const int kk = blockIdx.y;
  const double k = kv[kk];
  const int64_t m = (int64_t)blockIdx.x * FT + threadIdx.x;
  const bool active = m < M;
  double p[3] = {0, 0, 0}, x0[3] = {0, 0, 0}, nu0[3] = {0, 0, 1};
  cd P0 = {0, 0}, Pn0 = {0, 0};
  if (active) {
    for (int d = 0; d < 3; ++d) {
      p[d] = xp[3 * m + d];
      x0[d] = foot[8 * m + d];
      nu0[d] = foot[8 * m + 3 + d];
    }
    const double fxi = foot[8 * m + 6], feta = foot[8 * m + 7];
    const double L1 = 1.0 - fxi - feta;
    const double Nv[6] = {L1 * (2 * L1 - 1), fxi * (2 * fxi - 1), feta * (2 * feta - 1), 4 * L1 * fxi, 4 * fxi * feta,
                          4 * feta * L1};
    const int32_t* el = elems + 6 * (int64_t)foot_elem[m];
    const cd* P = surf + (int64_t)kk * 2 * N;
    for (int a = 0; a < 6; ++a) {
      cd v = P[el[a]], w = P[N + el[a]];
      P0.re += Nv[a] * v.re; P0.im += Nv[a] * v.im;
      Pn0.re += Nv[a] * w.re; Pn0.im += Nv[a] * w.im;
    }
  }
  const cd* Pqk = Pq + (int64_t)kk * EQ;
  const cd* Pnqk = Pnq + (int64_t)kk * EQ;
  cd sum = {0, 0};
  for (int64_t t0 = 0; t0 < EQ; t0 += FT) {
    const int64_t t = t0 + threadIdx.x;
    if (t < EQ) {
      sx[threadIdx.x] = qgeo[GX * EQ + t]; sy[threadIdx.x] = qgeo[GY * EQ + t]; sz[threadIdx.x] = qgeo[GZ * EQ + t];
      snx[threadIdx.x] = qgeo[GNX * EQ + t]; sny[threadIdx.x] = qgeo[GNY * EQ + t]; snz[threadIdx.x] = qgeo[GNZ * EQ + t];
      sw[threadIdx.x] = qgeo[GWJ * EQ + t];
      sP[threadIdx.x] = Pqk[t];
      sPn[threadIdx.x] = Pnqk[t];
    }
    __syncthreads();
    const int cnt = (EQ - t0) < FT ? (int)(EQ - t0) : FT;
    if (active) {
      for (int u = 0; u < cnt; ++u) {
        const double nx = snx[u], ny = sny[u], nz = snz[u];
        // source x_p
        double rx = sx[u] - p[0], ry = sy[u] - p[1], rz = sz[u] - p[2];
        double R = sqrt(rx * rx + ry * ry + rz * rz), iR = 1.0 / R, kR = k * R, s, c;
        sincos(kR, &s, &c);
        double rn = (rx * nx + ry * ny + rz * nz) * iR * iR * iR;
        cd Gp = {c * iR, s * iR}, dGp = {(-c - s * kR) * rn, (c * kR - s) * rn};
        // source x0
        rx = sx[u] - x0[0]; ry = sy[u] - x0[1]; rz = sz[u] - x0[2];
        R = sqrt(rx * rx + ry * ry + rz * rz); iR = 1.0 / R; kR = k * R;
        sincos(kR, &s, &c);
        rn = (rx * nx + ry * ny + rz * nz) * iR * iR * iR;
        cd G0 = {c * iR, s * iR}, dG0 = {(-c - s * kR) * rn, (c * kR - s) * rn};
        // g, f about x0
        const double nr = nu0[0] * rx + nu0[1] * ry + nu0[2] * rz;
        double sa = k * nr, sg, cg;
        sincos(sa, &sg, &cg);
        double nn = nu0[0] * nx + nu0[1] * ny + nu0[2] * nz;
        double g = cg, f = k > 0.0 ? sg / k : nr, dg = -k * sg * nn, df = cg * nn;  // f -> nu0.r at k = 0
        cd Pt = {sP[u].re - P0.re * g - Pn0.re * f, sP[u].im - P0.im * g - Pn0.im * f};
        cd dPt = {sPn[u].re - P0.re * dg - Pn0.re * df, sPn[u].im - P0.im * dg - Pn0.im * df};
        cd a = cmul(Pt, csub(dGp, dG0)), b = cmul(csub(Gp, G0), dPt);
        sum.re += sw[u] * (a.re - b.re);
        sum.im += sw[u] * (a.im - b.im);
      }
    }
    __syncthreads();
  }
  if (active) {
    const double inv4pi = 1.0 / (4.0 * kPi);
    T[(int64_t)kk * M + m] = {P0.re + sum.re * inv4pi, P0.im + sum.im * inv4pi};
  }
}

// Evaluates nk wavenumbers: surf [nk][2][N] -> T [nk][M].  scratch >= 2 * nk * E * Q * 16 B.
int field64(bie_ctx* c, const double* kv, int nk, const cd* surf, const double* xp, int64_t M,
            const int32_t* foot_elem, const double* foot, cd* T, void* scratch) {
  const int64_t EQ = c->E * c->rule.Q;
  cd* Pq = (cd*)scratch;
  cd* Pnq = Pq + (int64_t)nk * EQ;
  dim3 gi((unsigned)((EQ + 255) / 256), nk);
  BIE_LAUNCH(k_interp_q64<<<gi, 256, 0, c->stream>>>(c->elems, c->N, c->E, c->rule.Q, c->qshape, surf, Pq, Pnq));
  if (M > 0) {
    dim3 gf((unsigned)((M + FT - 1) / FT), nk);
    BIE_LAUNCH(k_field64<<<gf, FT, 0, c->stream>>>(c->elems, c->N, EQ, c->qgeo, Pq, Pnq, surf, xp, M, foot_elem, foot, kv, T));
  }
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}


// ------------------------------------------------------------------------------------------
// Mixed precision: the same formula in FP32 with compensated accumulation.  ACC = true forms the
// three phases (k|x - x_p|, k|x - x0|, k nu0.(x - x0)) in float-float and reduces them modulo
// 2 pi before sincosf; ACC = false uses FP32 distances and the SFU sine/cosine after an FP32
// reduction.  Point table: asm32.cu's layout (x_hi[3], x_lo[3], nu[3], wJ).
// ------------------------------------------------------------------------------------------
struct TwoPi3f {
  float c1, c2, c3, inv;
};

__device__ __forceinline__ void cis_ff(ff a, const TwoPi3f& tp, float& c, float& s) {
  const float n = round_small(__fmul_rn(a.hi, tp.inv));
  const float h = __fmaf_rn(-n, tp.c1, a.hi);
  float t = __fmaf_rn(-n, tp.c2, a.lo);
  t = __fmaf_rn(-n, tp.c3, t);
  const ff u = ff_two_sum(h, t);
  float sh, ch;
  sincosf(u.hi, &sh, &ch);
  c = __fmaf_rn(-u.lo, sh, ch);
  s = __fmaf_rn(u.lo, ch, sh);
}

__device__ __forceinline__ void cis_fast(float t, const TwoPi3f& tp, float& c, float& s) {
  const float n = round_small(__fmul_rn(t, tp.inv));
  float u = __fmaf_rn(-n, tp.c1, t);
  u = __fmaf_rn(-n, tp.c2, u);
  __sincosf(u, &s, &c);
}

__global__ void k_interp_q32(const int32_t* __restrict__ elems, int64_t N, int64_t E, int Q,
                             const double* __restrict__ qshape, const cd* __restrict__ surf, cf* __restrict__ Pq,
                             cf* __restrict__ Pnq) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int kk = blockIdx.y;
  if (p >= E * Q) return;
  int64_t e = p / Q;
  int q = (int)(p % Q);
  const cd* P = surf + (int64_t)kk * 2 * N;
  const cd* Pn = P + N;
  cd a = {0, 0}, b = {0, 0};
  for (int t = 0; t < 6; ++t) {
    int32_t j = elems[6 * e + t];
    double sh = qshape[q * 6 + t];
    a.re += sh * P[j].re; a.im += sh * P[j].im;
    b.re += sh * Pn[j].re; b.im += sh * Pn[j].im;
  }
  Pq[(int64_t)kk * E * Q + p] = {(float)a.re, (float)a.im};
  Pnq[(int64_t)kk * E * Q + p] = {(float)b.re, (float)b.im};
}

template <bool ACC>
__global__ void __launch_bounds__(FT) k_field32(const int32_t* __restrict__ elems, int64_t N, int64_t EQ,
                                                const float* __restrict__ qtab, const cf* __restrict__ Pq,
                                                const cf* __restrict__ Pnq, const cd* __restrict__ surf,
                                                const double* __restrict__ xp, int64_t M,
                                                const int32_t* __restrict__ foot_elem, const double* __restrict__ foot,
                                                const double* __restrict__ kv, cd* __restrict__ T, TwoPi3f tp) {
  __shared__ float st[17][FT];
  const int kk = blockIdx.y;
  const ff k = ff_from_double(kv[kk]);
  const float kinv = kinv32(kv[kk]);
  const int64_t m = (int64_t)blockIdx.x * FT + threadIdx.x;
  const bool active = m < M;
  ff p[3] = {{0, 0}, {0, 0}, {0, 0}}, x0[3] = {{0, 0}, {0, 0}, {0, 0}}, nu0[3] = {{0, 0}, {0, 0}, {1, 0}};
  float P0r = 0, P0i = 0, Q0r = 0, Q0i = 0;
  if (active) {
    for (int d = 0; d < 3; ++d) {
      p[d] = ff_from_double(xp[3 * m + d]);
      x0[d] = ff_from_double(foot[8 * m + d]);
      nu0[d] = ff_from_double(foot[8 * m + 3 + d]);
    }
    const double fxi = foot[8 * m + 6], feta = foot[8 * m + 7];
    const double L1 = 1.0 - fxi - feta;
    const double Nv[6] = {L1 * (2 * L1 - 1), fxi * (2 * fxi - 1), feta * (2 * feta - 1), 4 * L1 * fxi, 4 * fxi * feta,
                          4 * feta * L1};
    const int32_t* el = elems + 6 * (int64_t)foot_elem[m];
    const cd* P = surf + (int64_t)kk * 2 * N;
    double a0 = 0, a1 = 0, b0 = 0, b1 = 0;
    for (int a = 0; a < 6; ++a) {
      cd v = P[el[a]], w = P[N + el[a]];
      a0 += Nv[a] * v.re; a1 += Nv[a] * v.im;
      b0 += Nv[a] * w.re; b1 += Nv[a] * w.im;
    }
    P0r = (float)a0; P0i = (float)a1; Q0r = (float)b0; Q0i = (float)b1;
  }
  const cf* Pqk = Pq + (int64_t)kk * EQ;
  const cf* Pnqk = Pnq + (int64_t)kk * EQ;
  ksum sr, si;
  for (int64_t t0 = 0; t0 < EQ; t0 += FT) {
    const int64_t t = t0 + threadIdx.x;
    if (t < EQ) {
#pragma unroll
      for (int u = 0; u < 13; ++u) st[u][threadIdx.x] = qtab[u * EQ + t];
      const cf a = Pqk[t], b = Pnqk[t];
      st[13][threadIdx.x] = a.re; st[14][threadIdx.x] = a.im;
      st[15][threadIdx.x] = b.re; st[16][threadIdx.x] = b.im;
    }
    __syncthreads();
    const int cnt = (EQ - t0) < FT ? (int)(EQ - t0) : FT;
    if (active) {
      for (int u = 0; u < cnt; ++u) {
        const ff qx = {st[0][u], st[3][u]}, qy = {st[1][u], st[4][u]}, qz = {st[2][u], st[5][u]};
        const float nx = st[6][u], ny = st[7][u], nz = st[8][u], wj = st[9][u];
        const ff rpx = ff_sub(qx, p[0]), rpy = ff_sub(qy, p[1]), rpz = ff_sub(qz, p[2]);
        const ff r0x = ff_sub(qx, x0[0]), r0y = ff_sub(qy, x0[1]), r0z = ff_sub(qz, x0[2]);
        float cp, sp, c0, s0, cg, sg, Rp, R0, rnp, rn0, nrh;
        if (ACC) {
          const ff nux = {nx, st[10][u]}, nuy = {ny, st[11][u]}, nuz = {nz, st[12][u]};
          rnp = ff_add(ff_add(ff_mul(rpx, nux), ff_mul(rpy, nuy)), ff_mul(rpz, nuz)).hi;
          rn0 = ff_add(ff_add(ff_mul(r0x, nux), ff_mul(r0y, nuy)), ff_mul(r0z, nuz)).hi;
          const ff Rpf = ff_sqrt(ff_add(ff_add(ff_sqr(rpx), ff_sqr(rpy)), ff_sqr(rpz)));
          const ff R0f = ff_sqrt(ff_add(ff_add(ff_sqr(r0x), ff_sqr(r0y)), ff_sqr(r0z)));
          const ff nr = ff_add(ff_add(ff_mul(nu0[0], r0x), ff_mul(nu0[1], r0y)), ff_mul(nu0[2], r0z));
          cis_ff(ff_mul(k, Rpf), tp, cp, sp);
          cis_ff(ff_mul(k, R0f), tp, c0, s0);
          cis_ff(ff_mul(k, nr), tp, cg, sg);
          nrh = nr.hi;
          Rp = Rpf.hi;
          R0 = R0f.hi;
        } else {
          Rp = sqrtf(rpx.hi * rpx.hi + rpy.hi * rpy.hi + rpz.hi * rpz.hi);
          R0 = sqrtf(r0x.hi * r0x.hi + r0y.hi * r0y.hi + r0z.hi * r0z.hi);
          const float nr = nu0[0].hi * r0x.hi + nu0[1].hi * r0y.hi + nu0[2].hi * r0z.hi;
          nrh = nr;
          cis_fast(k.hi * Rp, tp, cp, sp);
          cis_fast(k.hi * R0, tp, c0, s0);
          cis_fast(k.hi * nr, tp, cg, sg);
          rnp = rpx.hi * nx + rpy.hi * ny + rpz.hi * nz;
          rn0 = r0x.hi * nx + r0y.hi * ny + r0z.hi * nz;
        }
        const float iRp = 1.0f / Rp, iR0 = 1.0f / R0;
        const float kRp = k.hi * Rp, kR0 = k.hi * R0;
        rnp *= iRp * iRp * iRp;
        rn0 *= iR0 * iR0 * iR0;
        const float Gpr = cp * iRp, Gpi = sp * iRp, G0r = c0 * iR0, G0i = s0 * iR0;
        const float dGpr = (-cp - sp * kRp) * rnp, dGpi = (cp * kRp - sp) * rnp;
        const float dG0r = (-c0 - s0 * kR0) * rn0, dG0i = (c0 * kR0 - s0) * rn0;
        const float nn = nu0[0].hi * nx + nu0[1].hi * ny + nu0[2].hi * nz;
        const float g = cg, f = kinv != 0.f ? sg * kinv : nrh, dg = -k.hi * sg * nn, df = cg * nn;
        const float Ptr = st[13][u] - P0r * g - Q0r * f, Pti = st[14][u] - P0i * g - Q0i * f;
        const float dPr = st[15][u] - P0r * dg - Q0r * df, dPi = st[16][u] - P0i * dg - Q0i * df;
        const float ddr = dGpr - dG0r, ddi = dGpi - dG0i, gdr = Gpr - G0r, gdi = Gpi - G0i;
        const float tr = (Ptr * ddr - Pti * ddi) - (gdr * dPr - gdi * dPi);
        const float ti = (Ptr * ddi + Pti * ddr) - (gdr * dPi + gdi * dPr);
        sr.add(wj * tr);
        si.add(wj * ti);
      }
    }
    __syncthreads();
  }
  if (active) {
    const double inv4pi = 1.0 / (4.0 * kPi);
    T[(int64_t)kk * M + m] = {(double)P0r + sr.value() * inv4pi, (double)P0i + si.value() * inv4pi};
  }
}

// k-batched variant of the float-float kernel: each (point, quadrature point) pair's geometry --
// the float-float distances to x_p and x0, nu0.(x - x0), r.nu -- is formed once and reused for FKB
// wavenumbers; per wavenumber only the three phases (float-float product reduced by pi/2 in one
// step, cis_ffprod) and the FP32 integrand remain.
constexpr int FKB = 8;

__global__ void __launch_bounds__(FT) k_field32b(const int32_t* __restrict__ elems, int64_t N, int64_t EQ,
                                                 const float* __restrict__ qtab, const cf* __restrict__ Pq,
                                                 const cf* __restrict__ Pnq, const cd* __restrict__ surf,
                                                 const double* __restrict__ xp, int64_t M,
                                                 const int32_t* __restrict__ foot_elem,
                                                 const double* __restrict__ foot, const double* __restrict__ kv,
                                                 int nk, cd* __restrict__ T, TwoPi3f tp, int uniform,
                                                 ff dk) {
  __shared__ float sg[13][FT];        // quadrature geometry tile
  __shared__ float sq[FKB][4][FT];    // Pq, Pnq (re, im) of the tile for each wavenumber
  __shared__ float s0[FKB][4][FT];    // P0, P0' (re, im) of each thread's point for each wavenumber
  __shared__ float sk[FKB][3];        // k (hi, lo), 1/k
  const int kbase = blockIdx.y * FKB;
  const int nkb = min(FKB, nk - kbase);
  const int tid = threadIdx.x;
  const int64_t m = (int64_t)blockIdx.x * FT + tid;
  const bool active = m < M;
  if (tid < nkb) {
    const ff k = ff_from_double(kv[kbase + tid]);
    sk[tid][0] = k.hi;
    sk[tid][1] = k.lo;
    sk[tid][2] = kinv32(kv[kbase + tid]);
  }
  ff p[3] = {{0, 0}, {0, 0}, {0, 0}}, x0[3] = {{0, 0}, {0, 0}, {0, 0}}, nu0[3] = {{0, 0}, {0, 0}, {1, 0}};
  if (active) {
    for (int d = 0; d < 3; ++d) {
      p[d] = ff_from_double(xp[3 * m + d]);
      x0[d] = ff_from_double(foot[8 * m + d]);
      nu0[d] = ff_from_double(foot[8 * m + 3 + d]);
    }
    const double fxi = foot[8 * m + 6], feta = foot[8 * m + 7];
    const double L1 = 1.0 - fxi - feta;
    const double Nv[6] = {L1 * (2 * L1 - 1), fxi * (2 * fxi - 1), feta * (2 * feta - 1), 4 * L1 * fxi, 4 * fxi * feta,
                          4 * feta * L1};
    const int32_t* el = elems + 6 * (int64_t)foot_elem[m];
    for (int j = 0; j < nkb; ++j) {
      const cd* P = surf + (int64_t)(kbase + j) * 2 * N;
      double a0 = 0, a1 = 0, b0 = 0, b1 = 0;
      for (int a = 0; a < 6; ++a) {
        const cd v = P[el[a]], w = P[N + el[a]];
        a0 += Nv[a] * v.re; a1 += Nv[a] * v.im;
        b0 += Nv[a] * w.re; b1 += Nv[a] * w.im;
      }
      s0[j][0][tid] = (float)a0; s0[j][1][tid] = (float)a1;
      s0[j][2][tid] = (float)b0; s0[j][3][tid] = (float)b1;
    }
  }
  ksum accr[FKB], acci[FKB];
  for (int64_t t0 = 0; t0 < EQ; t0 += FT) {
    const int64_t t = t0 + tid;
    __syncthreads();
    if (t < EQ) {
#pragma unroll
      for (int u = 0; u < 13; ++u) sg[u][tid] = qtab[u * EQ + t];
      for (int j = 0; j < nkb; ++j) {
        const cf a = Pq[(int64_t)(kbase + j) * EQ + t], b = Pnq[(int64_t)(kbase + j) * EQ + t];
        sq[j][0][tid] = a.re; sq[j][1][tid] = a.im;
        sq[j][2][tid] = b.re; sq[j][3][tid] = b.im;
      }
    }
    __syncthreads();
    const int cnt = (EQ - t0) < FT ? (int)(EQ - t0) : FT;
    if (!active) continue;
    for (int u = 0; u < cnt; ++u) {
      const ff qx = {sg[0][u], sg[3][u]}, qy = {sg[1][u], sg[4][u]}, qz = {sg[2][u], sg[5][u]};
      const float nx = sg[6][u], ny = sg[7][u], nz = sg[8][u], wj = sg[9][u];
      const ff nux = {nx, sg[10][u]}, nuy = {ny, sg[11][u]}, nuz = {nz, sg[12][u]};
      const ff rpx = ff_sub(qx, p[0]), rpy = ff_sub(qy, p[1]), rpz = ff_sub(qz, p[2]);
      const ff r0x = ff_sub(qx, x0[0]), r0y = ff_sub(qy, x0[1]), r0z = ff_sub(qz, x0[2]);
      const ff Rp = ff_sqrt(ff_add(ff_add(ff_sqr(rpx), ff_sqr(rpy)), ff_sqr(rpz)));
      const ff R0 = ff_sqrt(ff_add(ff_add(ff_sqr(r0x), ff_sqr(r0y)), ff_sqr(r0z)));
      const ff nr = ff_add(ff_add(ff_mul(nu0[0], r0x), ff_mul(nu0[1], r0y)), ff_mul(nu0[2], r0z));
      const float iRp = 1.0f / Rp.hi, iR0 = 1.0f / R0.hi;
      // x_p is off the surface (no cancellation in r.nu); x0 is on it, so r0.nu is second-order
      // small for nearby quadrature points and is formed in float-float
      const float rnp = (rpx.hi * nx + rpy.hi * ny + rpz.hi * nz) * iRp * iRp * iRp;
      const float rn0 = ff_add(ff_add(ff_mul(r0x, nux), ff_mul(r0y, nuy)), ff_mul(r0z, nuz)).hi * iR0 * iR0 * iR0;
      const float nn = nu0[0].hi * nx + nu0[1].hi * ny + nu0[2].hi * nz;
      // phase factors: on a uniform group k_j = k_0 + j dk, e^{i k_j R} = e^{i k_0 R} (e^{i dk R})^j with
      // both factors accurate and the powers taken by FP32 rotation (drift <= nkb ulps)
      float cp = 0.f, spp = 0.f, c0 = 0.f, s0v = 0.f, cg = 0.f, sgv = 0.f;
      float dcp = 1.f, dsp = 0.f, dc0 = 1.f, ds0 = 0.f, dcg = 1.f, dsg = 0.f;
      if (uniform) {
        const ff k0 = {sk[0][0], sk[0][1]};
        cis_ffprod(k0, Rp, cp, spp);
        cis_ffprod(k0, R0, c0, s0v);
        cis_ffprod(k0, nr, cg, sgv);
        cis_ffprod(dk, Rp, dcp, dsp);
        cis_ffprod(dk, R0, dc0, ds0);
        cis_ffprod(dk, nr, dcg, dsg);
      }
#pragma unroll
      for (int j = 0; j < FKB; ++j) {
        if (j < nkb) {
          const ff k = {sk[j][0], sk[j][1]};
          const float kinv = sk[j][2];
          if (!uniform) {
            cis_ffprod(k, Rp, cp, spp);
            cis_ffprod(k, R0, c0, s0v);
            cis_ffprod(k, nr, cg, sgv);
          } else if (j > 0) {
            float t = cp * dcp - spp * dsp;
            spp = spp * dcp + cp * dsp;
            cp = t;
            t = c0 * dc0 - s0v * ds0;
            s0v = s0v * dc0 + c0 * ds0;
            c0 = t;
            t = cg * dcg - sgv * dsg;
            sgv = sgv * dcg + cg * dsg;
            cg = t;
          }
          const float kRp = k.hi * Rp.hi, kR0 = k.hi * R0.hi;
          const float Gpr = cp * iRp, Gpi = spp * iRp, G0r = c0 * iR0, G0i = s0v * iR0;
          const float dGpr = (-cp - spp * kRp) * rnp, dGpi = (cp * kRp - spp) * rnp;
          const float dG0r = (-c0 - s0v * kR0) * rn0, dG0i = (c0 * kR0 - s0v) * rn0;
          const float g = cg, f = kinv != 0.f ? sgv * kinv : nr.hi, dg = -k.hi * sgv * nn, df = cg * nn;
          const float P0r = s0[j][0][tid], P0i = s0[j][1][tid], Q0r = s0[j][2][tid], Q0i = s0[j][3][tid];
          const float Ptr = sq[j][0][u] - P0r * g - Q0r * f, Pti = sq[j][1][u] - P0i * g - Q0i * f;
          const float dPr = sq[j][2][u] - P0r * dg - Q0r * df, dPi = sq[j][3][u] - P0i * dg - Q0i * df;
          const float ddr = dGpr - dG0r, ddi = dGpi - dG0i, gdr = Gpr - G0r, gdi = Gpi - G0i;
          const float tr = (Ptr * ddr - Pti * ddi) - (gdr * dPr - gdi * dPi);
          const float ti = (Ptr * ddi + Pti * ddr) - (gdr * dPi + gdi * dPr);
          accr[j].add(wj * tr);
          acci[j].add(wj * ti);
        }
      }
    }
  }
  if (active) {
    const double inv4pi = 1.0 / (4.0 * kPi);
    for (int j = 0; j < nkb; ++j)
      T[(int64_t)(kbase + j) * M + m] = {(double)s0[j][0][tid] + accr[j].value() * inv4pi,
                                         (double)s0[j][1][tid] + acci[j].value() * inv4pi};
  }
}

// Variant of k_field32b with the wavenumber-group size KB, the points per CTA TP and the minimum
// resident CTAs MINB as template parameters: terms are summed in FP32 over runs of 32 quadrature
// points and each run is added to a compensated sum kept in shared memory, so only 2 KB partial
// sums stay in registers; every phase (group start k_0 R and step dk R) comes from the
// float-float product reduced by pi/2 in one step (cis_ffprod).  far_r2: beyond it r0.nu_q is
// formed in FP32.
// ZF: the group may hold k = 0 (f takes its limit nu0.r there); false for groups of k > 0 only,
// which keeps the zero-frequency select out of the inner loop.
template <int KB, int TP, int MINB, int UT, bool ZF>
__global__ void __launch_bounds__(TP, MINB) k_field32c(const int32_t* __restrict__ elems, int64_t N, int64_t EQ,
                                                       const float* __restrict__ qtab, const cf* __restrict__ Pq,
                                                       const cf* __restrict__ Pnq, const cd* __restrict__ surf,
                                                       const double* __restrict__ xp, int64_t M,
                                                       const int32_t* __restrict__ foot_elem,
                                                       const double* __restrict__ foot, const double* __restrict__ kv,
                                                       int nk, cd* __restrict__ T, int uniform, ff dk,
                                                       float far_r2) {
  __shared__ float4 sg[UT][4];  // a tile of UT quadrature points: 13 table values (P32 order), padded
  __shared__ float4 sq[KB][UT];  // surface values at the tile's points: P re, im, dP re, im
  __shared__ float4 s0[KB][TP];  // surface values at the foot points, same order
  __shared__ float sacc[KB][4][TP];  // compensated sums: re (s, c), im (s, c)
  __shared__ float2 sk[KB];  // k (FP32 head), 1 / k (0 at k = 0)
  __shared__ float sklo[KB];  // k - head
  const int kbase = blockIdx.y * KB;
  const int nkb = min(KB, nk - kbase);
  const int tid = threadIdx.x;
  const int64_t m = (int64_t)blockIdx.x * TP + tid;
  const bool active = m < M;
  if (tid < nkb) {
    const ff k = ff_from_double(kv[kbase + tid]);
    sk[tid] = make_float2(k.hi, kinv32(kv[kbase + tid]));
    sklo[tid] = k.lo;
  }
#pragma unroll
  for (int j = 0; j < KB; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) sacc[j][q][tid] = 0.f;
  ff p[3] = {{0, 0}, {0, 0}, {0, 0}}, x0[3] = {{0, 0}, {0, 0}, {0, 0}}, nu0[3] = {{0, 0}, {0, 0}, {1, 0}};
  if (active) {
    for (int d = 0; d < 3; ++d) {
      p[d] = ff_from_double(xp[3 * m + d]);
      x0[d] = ff_from_double(foot[8 * m + d]);
      nu0[d] = ff_from_double(foot[8 * m + 3 + d]);
    }
    const double fxi = foot[8 * m + 6], feta = foot[8 * m + 7];
    const double L1 = 1.0 - fxi - feta;
    const double Nv[6] = {L1 * (2 * L1 - 1), fxi * (2 * fxi - 1), feta * (2 * feta - 1), 4 * L1 * fxi, 4 * fxi * feta,
                          4 * feta * L1};
    const int32_t* el = elems + 6 * (int64_t)foot_elem[m];
    for (int j = 0; j < nkb; ++j) {
      const cd* P = surf + (int64_t)(kbase + j) * 2 * N;
      double a0 = 0, a1 = 0, b0 = 0, b1 = 0;
      for (int a = 0; a < 6; ++a) {
        const cd v = P[el[a]], w = P[N + el[a]];
        a0 += Nv[a] * v.re; a1 += Nv[a] * v.im;
        b0 += Nv[a] * w.re; b1 += Nv[a] * w.im;
      }
      s0[j][tid] = make_float4((float)a0, (float)a1, (float)b0, (float)b1);
    }
  }
  float pr[KB], pim[KB];
#pragma unroll
  for (int j = 0; j < KB; ++j) pr[j] = pim[j] = 0.f;
  for (int64_t t0 = 0; t0 < EQ; t0 += UT) {
    const int cnt = (EQ - t0) < UT ? (int)(EQ - t0) : UT;
    __syncthreads();
    for (int e = tid; e < 13 * UT; e += TP) {  // consecutive threads, consecutive points
      const int f = e / UT, u = e - f * UT;
      if (u < cnt) reinterpret_cast<float*>(sg[u])[f] = qtab[f * EQ + t0 + u];
    }
    for (int e = tid; e < KB * UT; e += TP) {
      const int j = e / UT, u = e - j * UT;
      if (j < nkb && u < cnt) {
        const int64_t t = t0 + u;
        const cf a = Pq[(int64_t)(kbase + j) * EQ + t], b = Pnq[(int64_t)(kbase + j) * EQ + t];
        sq[j][u] = make_float4(a.re, a.im, b.re, b.im);
      }
    }
    __syncthreads();
    if (!active) continue;
    for (int u = 0; u < cnt; ++u) {
      const float4 g0 = sg[u][0], g1 = sg[u][1], g2 = sg[u][2], g3 = sg[u][3];
      const ff qx = {g0.x, g0.w}, qy = {g0.y, g1.x}, qz = {g0.z, g1.y};
      const float nx = g1.z, ny = g1.w, nz = g2.x, wj = g2.y;
      const ff nux = {nx, g2.z}, nuy = {ny, g2.w}, nuz = {nz, g3.x};
      // float-float geometry with lazy tails (distances, 1/R, nu0.r)
      const ff rpx = ff_diff_lazy(qx, p[0]), rpy = ff_diff_lazy(qy, p[1]), rpz = ff_diff_lazy(qz, p[2]);
      const ff r0x = ff_diff_lazy(qx, x0[0]), r0y = ff_diff_lazy(qy, x0[1]), r0z = ff_diff_lazy(qz, x0[2]);
      const ff R0sq = ff_norm2_lazy(r0x, r0y, r0z);
      float iRp, iR0;
      const ff Rp = ff_sqrt_lazy(ff_norm2_lazy(rpx, rpy, rpz), iRp);
      const ff R0 = ff_sqrt_lazy(R0sq, iR0);
      const ff nr = ff_dot3_lazy(nu0, r0x, r0y, r0z);
      // the recurrences below carry the weighted kernels Gp = w e^{ik Rp} / Rp and G0 (same for
      // the foot point); then dG/dnu = G (ik R - 1) r.nu / R^2
      const float ap = wj * iRp, a0 = wj * iR0;
      const float rnp = ((rpx.hi + rpx.lo) * nx + (rpy.hi + rpy.lo) * ny + (rpz.hi + rpz.lo) * nz) * iRp * iRp;
      // r0.nu is second-order small near the foot point (error-free products there); beyond
      // far_r2 its FP32 rounding eps R0 perturbs dG0 by eps / R0^2, the term's own rounding
      float rn0;
      if (R0sq.hi > far_r2) {
        rn0 = (r0x.hi + r0x.lo) * nx + (r0y.hi + r0y.lo) * ny + (r0z.hi + r0z.lo) * nz;
      } else {
        const ff nuq[3] = {nux, nuy, nuz};
        const ff d = ff_dot3_lazy(nuq, r0x, r0y, r0z);
        rn0 = d.hi + d.lo;
      }
      rn0 *= iR0 * iR0;
      const float nn = nu0[0].hi * nx + nu0[1].hi * ny + nu0[2].hi * nz;
      float cp = 0.f, spp = 0.f, c0 = 0.f, s0v = 0.f, cg = 0.f, sgv = 0.f;
      float dcp = 1.f, dsp = 0.f, dc0 = 1.f, ds0 = 0.f, dcg = 1.f, dsg = 0.f;
      if (uniform) {
        const ff k0 = {sk[0].x, sklo[0]};
        cis_ffprod(k0, Rp, cp, spp);
        cis_ffprod(k0, R0, c0, s0v);
        cis_ffprod(k0, nr, cg, sgv);
        // step phases dk R
        cis_ffprod(dk, Rp, dcp, dsp);
        cis_ffprod(dk, R0, dc0, ds0);
        cis_ffprod(dk, nr, dcg, dsg);
        cp *= ap; spp *= ap;
        c0 *= a0; s0v *= a0;
      }
#pragma unroll
      for (int j = 0; j < KB; ++j) {
        if (j < nkb) {
          const float2 kj = sk[j];
          const float khi = kj.x, kinv = kj.y;
          if (!uniform) {
            const ff k = {khi, sklo[j]};
            cis_ffprod(k, Rp, cp, spp);
            cis_ffprod(k, R0, c0, s0v);
            cis_ffprod(k, nr, cg, sgv);
            cp *= ap; spp *= ap;
            c0 *= a0; s0v *= a0;
          } else if (j > 0) {
            float t = cp * dcp - spp * dsp;
            spp = spp * dcp + cp * dsp;
            cp = t;
            t = c0 * dc0 - s0v * ds0;
            s0v = s0v * dc0 + c0 * ds0;
            c0 = t;
            t = cg * dcg - sgv * dsg;
            sgv = sgv * dcg + cg * dsg;
            cg = t;
          }
          const float kRp = khi * Rp.hi, kR0 = khi * R0.hi;
          // G weighted by w; dG/dnu = -(Gr + Gi kR) rn + i (Gr kR - Gi) rn, taken as the
          // difference dGp - dG0 directly
          const float gdr = cp - c0, gdi = spp - s0v;
          const float ddr = __fmaf_rn(__fmaf_rn(s0v, kR0, c0), rn0, -(__fmaf_rn(spp, kRp, cp) * rnp));
          const float ddi = __fmaf_rn(__fmaf_rn(cp, kRp, -spp), rnp, -(__fmaf_rn(c0, kR0, -s0v) * rn0));
          // f = sin(k nu0.r)/k, or its limit nu0.r at k = 0 (kinv 0)
          const float g = cg, f = (ZF && kinv == 0.f) ? nr.hi : sgv * kinv, dg = -khi * sgv * nn, df = cg * nn;
          const float4 p0 = s0[j][tid], pq = sq[j][u];
          const float P0r = p0.x, P0i = p0.y, Q0r = p0.z, Q0i = p0.w;
          const float Ptr = pq.x - P0r * g - Q0r * f, Pti = pq.y - P0i * g - Q0i * f;
          const float dPr = pq.z - P0r * dg - Q0r * df, dPi = pq.w - P0i * dg - Q0i * df;
          // run sums of w [P~ (dGp - dG0) - (Gp - G0) dP~]
          float a = __fmaf_rn(Ptr, ddr, pr[j]);
          a = __fmaf_rn(-Pti, ddi, a);
          a = __fmaf_rn(-gdr, dPr, a);
          pr[j] = __fmaf_rn(gdi, dPi, a);
          a = __fmaf_rn(Ptr, ddi, pim[j]);
          a = __fmaf_rn(Pti, ddr, a);
          a = __fmaf_rn(-gdr, dPi, a);
          pim[j] = __fmaf_rn(-gdi, dPr, a);
        }
      }
      if ((u & 31) == 31 || u == cnt - 1) {  // add the run to the compensated sums
#pragma unroll
        for (int j = 0; j < KB; ++j) {
          if (j < nkb) {
            ff a = ff_two_sum(sacc[j][0][tid], pr[j]);
            sacc[j][0][tid] = a.hi;
            sacc[j][1][tid] += a.lo;
            a = ff_two_sum(sacc[j][2][tid], pim[j]);
            sacc[j][2][tid] = a.hi;
            sacc[j][3][tid] += a.lo;
          }
          pr[j] = pim[j] = 0.f;
        }
      }
    }
  }
  if (active) {
    const double inv4pi = 1.0 / (4.0 * kPi);
    for (int j = 0; j < nkb; ++j) {
      const double sr = (double)sacc[j][0][tid] + (double)sacc[j][1][tid];
      const double si = (double)sacc[j][2][tid] + (double)sacc[j][3][tid];
      T[(int64_t)(kbase + j) * M + m] = {(double)s0[j][tid].x + sr * inv4pi, (double)s0[j][tid].y + si * inv4pi};
    }
  }
}

double far_radius2(bie_ctx* c);

template <int KB, int TP, int MINB, int UT>
static void launch_field32c(bie_ctx* c, int64_t EQ, const cf* Pq, const cf* Pnq, const cd* surf, const double* xp,
                            int64_t M, const int32_t* foot_elem, const double* foot, const double* kv, int nk, cd* T,
                            TwoPi3f tp, int uniform, ff dk, bool zero) {
  (void)tp;
  dim3 gb((unsigned)((M + TP - 1) / TP), (unsigned)((nk + KB - 1) / KB));
  const float far_r2 = (float)far_radius2(c);
  if (zero)
    BIE_LAUNCH(k_field32c<KB, TP, MINB, UT, true><<<gb, TP, 0, c->stream>>>(
        c->elems, c->N, EQ, c->qgeo32, Pq, Pnq, surf, xp, M, foot_elem, foot, kv, nk, T, uniform, dk, far_r2));
  else
    BIE_LAUNCH(k_field32c<KB, TP, MINB, UT, false><<<gb, TP, 0, c->stream>>>(
        c->elems, c->N, EQ, c->qgeo32, Pq, Pnq, surf, xp, M, foot_elem, foot, kv, nk, T, uniform, dk, far_r2));
}

int ensure_mixed_tables(bie_ctx* c);

int field_mixed(bie_ctx* c, const double* kv, int nk, const cd* surf, const double* xp, int64_t M,
                const int32_t* foot_elem, const double* foot, cd* T, void* scratch, size_t scratch_bytes) {
  BIE_TRY(ensure_mixed_tables(c));
  const int64_t EQ = c->E * c->rule.Q;
  if ((size_t)2 * nk * EQ * sizeof(cf) > scratch_bytes) return fail(BIE_ERR_STATE, "field scratch too small");
  cf* Pq = (cf*)scratch;
  cf* Pnq = Pq + (int64_t)nk * EQ;
  dim3 gi((unsigned)((EQ + 255) / 256), nk);
  BIE_LAUNCH(k_interp_q32<<<gi, 256, 0, c->stream>>>(c->elems, c->N, c->E, c->rule.Q, c->qshape, surf, Pq, Pnq));
  TwoPi3f tp;
  const double two_pi = 2.0 * kPi;
  tp.c1 = (float)two_pi;
  tp.c2 = (float)(two_pi - (double)tp.c1);
  tp.c3 = (float)((two_pi - (double)tp.c1 - (double)tp.c2) + 2.4492935982947064e-16);
  tp.inv = (float)(1.0 / two_pi);
  if (M > 0) {
    dim3 gf((unsigned)((M + FT - 1) / FT), nk);
    if (c->field_accurate_phase) {
      const int v = c->field_variant;
      std::vector<double> hk(nk);
      BIE_CUDA_TRY(cudaMemcpyAsync(hk.data(), kv, nk * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
      // Segments of the wavenumber list, one launch each: maximal runs of equally spaced
      // wavenumbers (at least 4) take the phase recurrence inside their groups of KB, the rest
      // runs without it -- so that a sweep with the zero-frequency term in front (or any
      // uniform runs inside a list) keeps the recurrence where it applies.
      std::vector<std::pair<int, int>> segs;  // (start, length); a negative length: no recurrence
      {
        int i = 0, nu_start = -1;
        while (i < nk) {
          int L = 1;
          if (i + 1 < nk) {
            const double d = hk[i + 1] - hk[i];
            L = 2;
            if (!(d > 0.0)) L = 1;
            else
              while (i + L < nk && std::fabs(hk[i + L] - (hk[i] + L * d)) <= 1e-12 * std::fabs(hk[i + L])) ++L;
          }
          if (L >= 4) {
            if (nu_start >= 0) { segs.push_back({nu_start, -(i - nu_start)}); nu_start = -1; }
            segs.push_back({i, L});
            i += L;
          } else {
            if (nu_start < 0) nu_start = i;
            ++i;
          }
        }
        if (nu_start >= 0) segs.push_back({nu_start, -(nk - nu_start)});
      }
      for (const auto& sg : segs) {
        const int r0 = sg.first, n = sg.second > 0 ? sg.second : -sg.second;
        const int uniform = sg.second > 0 ? 1 : 0;
        const double dkv = uniform ? hk[r0 + 1] - hk[r0] : 0.0;
        // k = 0 (the zero-frequency term) takes f's limit inside the kernel; launches without it
        // keep that select out of the inner loop
        bool zero_s = false;
        for (int j = 0; j < n; ++j) zero_s |= hk[r0 + j] == 0.0;
        const ff dkf = ff_from_double(dkv);
        const double* kr = kv + r0;
        const cf *Pqr = Pq + (int64_t)r0 * EQ, *Pnqr = Pnq + (int64_t)r0 * EQ;
        const cd* sr = surf + (int64_t)r0 * 2 * c->N;
        cd* Tr = T + (int64_t)r0 * M;
        if (v == 1) {
          launch_field32c<16, 64, 4, 64>(c, EQ, Pqr, Pnqr, sr, xp, M, foot_elem, foot, kr, n, Tr, tp, uniform, dkf, zero_s);
        } else if (v == 2) {
          launch_field32c<16, 128, 3, 32>(c, EQ, Pqr, Pnqr, sr, xp, M, foot_elem, foot, kr, n, Tr, tp, uniform, dkf, zero_s);
        } else {
          dim3 gb((unsigned)((M + FT - 1) / FT), (unsigned)((n + FKB - 1) / FKB));
          BIE_LAUNCH(k_field32b<<<gb, FT, 0, c->stream>>>(c->elems, c->N, EQ, c->qgeo32, Pqr, Pnqr, sr, xp, M, foot_elem,
                                                          foot, kr, n, Tr, tp, uniform, dkf));
        }
      }
    }
    else
      BIE_LAUNCH(k_field32<false><<<gf, FT, 0, c->stream>>>(c->elems, c->N, EQ, c->qgeo32, Pq, Pnq, surf, xp, M, foot_elem,
                                                 foot, kv, T, tp));
  }
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

}  // namespace bie
