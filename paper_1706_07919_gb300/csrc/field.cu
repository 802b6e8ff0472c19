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
        double sa = k * (nu0[0] * rx + nu0[1] * ry + nu0[2] * rz), sg, cg;
        sincos(sa, &sg, &cg);
        double nn = nu0[0] * nx + nu0[1] * ny + nu0[2] * nz;
        double g = cg, f = sg / k, dg = -k * sg * nn, df = cg * nn;
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
  k_interp_q64<<<gi, 256, 0, c->stream>>>(c->elems, c->N, c->E, c->rule.Q, c->qshape, surf, Pq, Pnq);
  if (M > 0) {
    dim3 gf((unsigned)((M + FT - 1) / FT), nk);
    k_field64<<<gf, FT, 0, c->stream>>>(c->elems, c->N, EQ, c->qgeo, Pq, Pnq, surf, xp, M, foot_elem, foot, kv, T);
  }
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

}  // namespace bie
