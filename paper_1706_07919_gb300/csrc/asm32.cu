// asm32.cu -- FP32 assembly of Eq. (BRIEF) for the mixed-precision path (same system as
// asm64.cu; see there for the row equation and the bulk/near split).
//
// Precision plan (each matrix entry to about FP32 rounding, independent of k R):
//   * positions and node normals are float-float (hi + lo), so x_q - x_i, |x_q - x_i| and
//     nu_i.(x_q - x_i) carry ~48 bits;
//   * both phases (k R for G, k nu_i.r for g and f) are formed and reduced modulo 2 pi in
//     float-float, then sincosf of the FP32 head plus a first-order correction by the tail;
//   * amplitudes (1/R, r.nu/R^3, w J N_a) are FP32;
//   * the row sums alpha_i, beta_i and b_i (over all E*Q points, with cancellation) are
//     compensated (Kahan-Babuska-Neumaier) sums.
// Output: A as interleaved complex FP32 [N][ld], b as complex FP64 [N].
#include <algorithm>

#include "bie_common.cuh"

namespace bie {

// Mixed-path point table: SoA of 13 floats per point:
//   x_hi, y_hi, z_hi, x_lo, y_lo, z_lo, nx, ny, nz, wJ, nx_lo, ny_lo, nz_lo
// (the normal's low parts let r.nu, a second-order small quantity for nearby points on one smooth
// surface, be formed in float-float).
enum { P32XH = 0, P32YH, P32ZH, P32XL, P32YL, P32ZL, P32NX, P32NY, P32NZ, P32W, P32NXL, P32NYL, P32NZL, P32COUNT };

// aos (optional): the same 13 values per point as one 64-byte record [n][16 floats].
__global__ void k_points_to32(const double* __restrict__ g, int64_t n, float* __restrict__ o,
                              float4* __restrict__ aos) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  float v[P32COUNT];
  for (int d = 0; d < 3; ++d) {
    const ff x = ff_from_double(g[(GX + d) * n + p]);
    const ff nv = ff_from_double(g[(GNX + d) * n + p]);
    v[P32XH + d] = x.hi; v[P32XL + d] = x.lo;
    v[P32NX + d] = nv.hi; v[P32NXL + d] = nv.lo;
  }
  v[P32W] = (float)g[GWJ * n + p];
  for (int f = 0; f < P32COUNT; ++f) o[f * n + p] = v[f];
  if (aos) {
    float4* a = aos + p * 4;
    a[0] = make_float4(v[0], v[1], v[2], v[3]);
    a[1] = make_float4(v[4], v[5], v[6], v[7]);
    a[2] = make_float4(v[8], v[9], v[10], v[11]);
    a[3] = make_float4(v[12], 0.f, 0.f, 0.f);
  }
}

// The bulk kernel's copy of the same table, re-ordered for coalesced loads: elements in colour
// order (position t of the colour-sorted list) and point-major, index (f * Q + q) * E + t, so
// that the lanes of a warp -- consecutive elements of one colour -- read consecutive floats.
// Element connectivity in the same order: esort[a * E + t].
__global__ void k_points_to32_sorted(const double* __restrict__ g, const int32_t* __restrict__ perm,
                                     const int32_t* __restrict__ elems, int64_t E, int Q, float* __restrict__ o,
                                     int32_t* __restrict__ esort, float4* __restrict__ aos) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= E * Q) return;
  const int64_t t = idx % E;
  const int q = (int)(idx / E);
  const int64_t e = perm[t];
  const int64_t n = E * Q, src = e * Q + q;
  float v[P32COUNT];
  for (int d = 0; d < 3; ++d) {
    const ff x = ff_from_double(g[(GX + d) * n + src]);
    const ff nv = ff_from_double(g[(GNX + d) * n + src]);
    v[P32XH + d] = x.hi; v[P32XL + d] = x.lo;
    v[P32NX + d] = nv.hi; v[P32NXL + d] = nv.lo;
  }
  const ff w = ff_from_double(g[GWJ * n + src]);
  v[P32W] = w.hi;
  for (int f = 0; f < P32COUNT; ++f) o[((int64_t)f * Q + q) * E + t] = v[f];
  // the same 13 values as one 64-byte record, then the weight's low part (float-float kernels)
  float4* a = aos + ((int64_t)q * E + t) * 4;
  a[0] = make_float4(v[0], v[1], v[2], v[3]);
  a[1] = make_float4(v[4], v[5], v[6], v[7]);
  a[2] = make_float4(v[8], v[9], v[10], v[11]);
  a[3] = make_float4(v[12], w.lo, 0.f, 0.f);
  if (q == 0)
    for (int a = 0; a < 6; ++a) esort[a * E + t] = elems[6 * e + a];
}

// 2 pi as an unevaluated sum of three floats, and 1 / (2 pi).
struct TwoPi3 {
  float c1, c2, c3, inv;
};

struct Kern32 {
  float Gr, Gi, dGr, dGi;
  float alr, ali, ber, bei;  // g dG - dg G, f dG - df G (without w J)
};

// far_r2: beyond R^2 > far_r2 (a few element sizes) r.nu_q is formed in FP32: its absolute error
// eps R then perturbs dG by eps / R^2, the entry's own rounding.
__device__ __forceinline__ void kernel32(const ff k, const float kinv, const ff* xi, const ff* nui, const TwoPi3& tp,
                                         const float* q, Kern32& o, float far_r2 = 3.0e38f) {
  // r = x_q - x_i in float-float
  const ff rx = ff_diff_lazy(ff{q[0], q[3]}, xi[0]);
  const ff ry = ff_diff_lazy(ff{q[1], q[4]}, xi[1]);
  const ff rz = ff_diff_lazy(ff{q[2], q[5]}, xi[2]);
  const ff R2 = ff_norm2_lazy(rx, ry, rz);
  float invR;
  const ff R = ff_sqrt_lazy(R2, invR);
  const ff nr = ff_dot3_lazy(nui, rx, ry, rz);
  float c, s;
  cis_ffprod(k, R, c, s);
  const float kR = k.hi * R.hi;
  o.Gr = c * invR;
  o.Gi = s * invR;
  float rnu;
  if (R2.hi > far_r2) {
    rnu = (rx.hi + rx.lo) * q[6] + (ry.hi + ry.lo) * q[7] + (rz.hi + rz.lo) * q[8];
  } else {
    const ff nq[3] = {ff{q[6], q[10]}, ff{q[7], q[11]}, ff{q[8], q[12]}};
    const ff d = ff_dot3_lazy(nq, rx, ry, rz);
    rnu = d.hi + d.lo;
  }
  const float rn = rnu * invR * invR * invR;
  o.dGr = (-c - s * kR) * rn;
  o.dGi = (c * kR - s) * rn;
  float cg, sg;
  cis_ffprod(k, nr, cg, sg);
  const float nn = nui[0].hi * q[6] + nui[1].hi * q[7] + nui[2].hi * q[8];
  const float g = cg, f = kinv != 0.f ? sg * kinv : nr.hi, dg = -k.hi * sg * nn, df = cg * nn;
  o.alr = g * o.dGr - dg * o.Gr;
  o.ali = g * o.dGi - dg * o.Gi;
  o.ber = f * o.dGr - df * o.Gr;
  o.bei = f * o.dGi - df * o.Gi;
}

struct RowSums {
  ksum ar, ai, br, bi, sr, si;
};

__device__ __forceinline__ void load_point(const float* __restrict__ tab, int64_t n, int64_t p, float* q) {
#pragma unroll
  for (int t = 0; t < P32COUNT; ++t) q[t] = tab[t * n + p];
}

// grid: (ceil(N / rows), nk); block: 32 * rows * W (W warps share a row: the elements of one
// colour share no node, so they can scatter into the row concurrently; colours are separated by
// a barrier of the row's warps); dynamic smem: rows * N * sizeof(cf)
constexpr int ASM_W = 2;
__global__ void __launch_bounds__(512) k_asm32_bulk(
    const double* __restrict__ nodes, const double* __restrict__ normals, const uint8_t* __restrict__ bc,
    const int32_t* __restrict__ esort, int64_t N, int64_t E, int Q, const float* __restrict__ qtab,
    const float* __restrict__ qshape, const int32_t* __restrict__ color_off, int ncolors,
    const double* __restrict__ kv, const cd* __restrict__ known,
    cf* __restrict__ A, int64_t lda, double* __restrict__ rowsum /* [nk][N][6] */, int rows, TwoPi3 tp,
    float far_r2) {
  extern __shared__ cf acc32[];
  __shared__ float shp[64 * 6];
  __shared__ double part[16][ASM_W][6];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rw = warp / ASM_W, sub = warp % ASM_W;
  const int kk = blockIdx.y;
  const ff k = ff_from_double(kv[kk]);
  const float kinv = kinv32(kv[kk]);
  for (int t = threadIdx.x; t < Q * 6; t += blockDim.x) shp[t] = qshape[t];
  for (int64_t t = threadIdx.x; t < (int64_t)rows * N; t += blockDim.x) acc32[t] = {0.f, 0.f};
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * rows + rw;
  const bool valid = i < N;
  cf* row = acc32 + (int64_t)rw * N;
  const cd* kn = known + (int64_t)kk * N;
  ff xi[3], nui[3];
  for (int d = 0; d < 3; ++d) {
    xi[d] = ff_from_double(valid ? nodes[3 * i + d] : 0.0);
    nui[d] = ff_from_double(valid ? normals[3 * i + d] : 0.0);
  }
  RowSums S;
  for (int col = 0; col < ncolors; ++col) {
    for (int32_t t = color_off[col] + sub * 32 + lane; valid && t < color_off[col + 1]; t += 32 * ASM_W) {
      int32_t el[6];
      bool near = false;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        el[a] = esort[a * E + t];  // `elems` in colour order (k_points_to32_sorted)
        near |= (el[a] == i);
      }
      if (near) continue;
      float hr[6], hi[6], gr[6], gi[6];
#pragma unroll
      for (int a = 0; a < 6; ++a) { hr[a] = hi[a] = gr[a] = gi[a] = 0.f; }
      // the element's share of the row sums in FP32 (Q terms), then one compensated addition each
      float ear = 0.f, eai = 0.f, ebr = 0.f, ebi = 0.f;
      for (int qq = 0; qq < Q; ++qq) {
        float q[P32COUNT];
#pragma unroll
        for (int f = 0; f < P32COUNT; ++f) q[f] = qtab[((int64_t)f * Q + qq) * E + t];
        Kern32 K;
        kernel32(k, kinv, xi, nui, tp, q, K, far_r2);
        const float wj = q[P32W];
        ear = __fmaf_rn(wj, K.alr, ear); eai = __fmaf_rn(wj, K.ali, eai);
        ebr = __fmaf_rn(wj, K.ber, ebr); ebi = __fmaf_rn(wj, K.bei, ebi);
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          const float cw = wj * shp[qq * 6 + a];
          hr[a] = __fmaf_rn(cw, K.dGr, hr[a]); hi[a] = __fmaf_rn(cw, K.dGi, hi[a]);
          gr[a] = __fmaf_rn(cw, K.Gr, gr[a]);  gi[a] = __fmaf_rn(cw, K.Gi, gi[a]);
        }
      }
      S.ar.add(ear); S.ai.add(eai);
      S.br.add(ebr); S.bi.add(ebi);
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const int32_t j = el[a];
        const float kr = (float)kn[j].re, ki = (float)kn[j].im;
        if (bc[j] == 0) {  // hard column: A += H, b += Gm P'_known
          row[j].re += hr[a]; row[j].im += hi[a];
          S.sr.add(gr[a] * kr - gi[a] * ki); S.si.add(gr[a] * ki + gi[a] * kr);
        } else {           // soft column: A -= Gm, b -= H P_known
          row[j].re -= gr[a]; row[j].im -= gi[a];
          S.sr.add(-(hr[a] * kr - hi[a] * ki)); S.si.add(-(hr[a] * ki + hi[a] * kr));
        }
      }
    }
    bar_named(1 + rw, 32 * ASM_W);  // the row's warps finish the colour (rows <= 8: ids 1..8)
  }
  // reduce the compensated sums across the warp in FP64 (12 values per row)
  double v[12] = {(double)S.ar.s, (double)S.ar.c, (double)S.ai.s, (double)S.ai.c, (double)S.br.s, (double)S.br.c,
                  (double)S.bi.s, (double)S.bi.c, (double)S.sr.s, (double)S.sr.c, (double)S.si.s, (double)S.si.c};
  double out[6];
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    double x = v[2 * t] + v[2 * t + 1];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    out[t] = x;
  }
  if (lane == 0)
    for (int t = 0; t < 6; ++t) part[rw][sub][t] = out[t];
  __syncthreads();
  if (!valid) return;
  cf* Arow = A + ((int64_t)kk * N + i) * lda;
  for (int64_t j = sub * 32 + lane; j < N; j += 32 * ASM_W) Arow[j] = row[j];
  if (sub == 0 && lane == 0) {
    double* rs = rowsum + ((int64_t)kk * N + i) * 6;
    for (int t = 0; t < 6; ++t) {
      double v = 0.0;
      for (int w = 0; w < ASM_W; ++w) v += part[rw][w][t];
      rs[t] = v;
    }
  }
}

// Known boundary values at the quadrature points of the colour-sorted elements:
//   kq[k][qq][t] = sum_a N_a(q_qq) known[k][el_t[a]]  (FP32 complex)
// so that an element whose six nodes share one boundary condition adds its right-hand-side share
// as sum_q w_q K_q kq_q (K = G on a hard element, -dG/dnu on a soft one) instead of carrying the
// six nodal sums of both kernels.  grid (ceil(E / 256), nk), block 256.
__global__ void k_known_q32(const int32_t* __restrict__ esort, int64_t E, int Q, const float* __restrict__ qshape,
                            const cd* __restrict__ known, int64_t N, cf* __restrict__ kq) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int kk = blockIdx.y;
  if (t >= E) return;
  cd kn[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) kn[a] = known[(int64_t)kk * N + esort[a * E + t]];
  for (int qq = 0; qq < Q; ++qq) {
    double sr = 0.0, si = 0.0;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      const double sh = qshape[qq * 6 + a];
      sr += sh * kn[a].re;
      si += sh * kn[a].im;
    }
    kq[((int64_t)kk * Q + qq) * E + t] = {(float)sr, (float)si};
  }
}

// Bulk assembly for meshes whose elements each carry one boundary condition on all six nodes
// (every element of a sound-hard or sound-soft body), KB wavenumbers per thread: the geometry of
// a (row, quadrature point) pair -- float-float r, R, nu_i.r, r.nu_q -- is formed once and used
// for KB wavenumbers, each with its own float-float phases (no recurrence: every entry keeps the
// accuracy of the one-wavenumber kernel).  Per element and wavenumber a lane carries the six nodal
// sums of the one kernel that enters A (dG/dnu on a hard element, -G on a soft one), the
// right-hand-side sum against the interpolated known values kq, and the two regularisation sums.
// A row has ASM_W x QS warps: ASM_W warps take consecutive elements of a colour and, with QS = 2,
// a second set of ASM_W warps takes the other half of the same elements' quadrature points, so
// that the registers of KB = 2 fit 16 warps per SM; the halves add into the row one after the
// other (barrier of the row's warps in between: fixed order, deterministic sums).
// grid (ceil(N / rows), ceil(nk / KB)); block 32 * rows * ASM_W * QS.  Where a row accumulates:
//   MODE 0: shared memory, rows * KB * N cf;
//   MODE 1 (large N): A itself, each row owned by one CTA and the row's warps ordered by the same
//     barriers (scattered read-modify-writes in L2);
//   MODE 2 (large N cut into column windows, see build_colouring): shared memory, rows * KB * ws
//     cf, one window of columns after the other -- the window's elements of every colour, then the
//     window copied to A -- so that each entry of A is written once.
template <int KB, int QS, int MODE>
__global__ void __launch_bounds__(256, 2) k_asm32_bulk_u(
    const double* __restrict__ nodes, const double* __restrict__ normals, const uint8_t* __restrict__ bc,
    const int32_t* __restrict__ esort, int64_t N, int64_t E, int Q, const float4* __restrict__ qaos,
    const float* __restrict__ qshape, const int32_t* __restrict__ color_off, int ncolors,
    const double* __restrict__ kv, int nk, const cf* __restrict__ kq, cf* __restrict__ A, int64_t lda,
    double* __restrict__ rowsum /* [nk][N][6] */, int rows, TwoPi3 tp, float far_r2,
    const int32_t* __restrict__ win_lo, const int32_t* __restrict__ wcol_off, int nwin, int ws) {
  constexpr bool GROW = MODE == 1;
  constexpr int WR = ASM_W * QS;  // warps per row
  extern __shared__ cf acc32[];
  __shared__ float shp[64 * 6];
  __shared__ double part[8][WR][KB][6];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rw = warp / WR, wr = warp % WR, sub = wr % ASM_W, h = wr / ASM_W;
  const int k0 = blockIdx.y * KB;
  const int nkb = min(KB, nk - k0);
  ff k[KB];
  float kinv[KB];
#pragma unroll
  for (int j = 0; j < KB; ++j) {
    const int kj = min(k0 + j, nk - 1);  // a ragged last group repeats its last wavenumber
    k[j] = ff_from_double(kv[kj]);
    kinv[j] = kinv32(kv[kj]);
  }
  for (int t = threadIdx.x; t < Q * 6; t += blockDim.x) shp[t] = qshape[t];
  const int64_t i = (int64_t)blockIdx.x * rows + rw;
  const bool valid = i < N;
  // row j of this CTA's row rw: in shared memory, or (GROW) row i of system k0 + j in A
  auto row_of = [&](int j) -> cf* {
    if constexpr (GROW) return A + ((int64_t)(k0 + j) * N + i) * lda;
    else if constexpr (MODE == 2) return acc32 + ((int64_t)rw * KB + j) * ws;
    else return acc32 + ((int64_t)rw * KB + j) * N;
  };
  if constexpr (GROW) {
    if (valid)
      for (int j = 0; j < nkb; ++j) {
        cf* r = row_of(j);
        for (int64_t c2 = wr * 32 + lane; c2 < N; c2 += 32 * WR) r[c2] = {0.f, 0.f};
      }
  } else if constexpr (MODE == 0) {
    for (int64_t t = threadIdx.x; t < (int64_t)rows * KB * N; t += blockDim.x) acc32[t] = {0.f, 0.f};
  }
  __syncthreads();
  const int qlo = h * Q / QS, qhi = (h + 1) * Q / QS;
  ff xi[3], nui[3];
  for (int d = 0; d < 3; ++d) {
    xi[d] = ff_from_double(valid ? nodes[3 * i + d] : 0.0);
    nui[d] = ff_from_double(valid ? normals[3 * i + d] : 0.0);
  }
  RowSums S[KB];
  const int nw = MODE == 2 ? nwin : 1;
  for (int w = 0; w < nw; ++w) {
  int w0 = 0;
  if constexpr (MODE == 2) {  // the row's window accumulator starts at zero
    w0 = win_lo[w];
    const int ww = win_lo[w + 1] - w0;
    for (int j = 0; j < KB; ++j) {
      cf* r = row_of(j);
      for (int c2 = wr * 32 + lane; c2 < ww; c2 += 32 * WR) r[c2] = {0.f, 0.f};
    }
    bar_named(1 + rw, 32 * WR);
  }
  for (int col = 0; col < ncolors; ++col) {
    int32_t cbeg, cend;
    if constexpr (MODE == 2) {
      cbeg = wcol_off[col * (nwin + 1) + w];
      cend = wcol_off[col * (nwin + 1) + w + 1];
    } else {
      cbeg = color_off[col];
      cend = color_off[col + 1];
    }
    // the same trip count for all warps of the row (the barriers below are the row's)
    const int iters = valid ? (cend - cbeg + 32 * ASM_W - 1) / (32 * ASM_W) : 0;
    for (int it = 0; it < iters; ++it) {
      const int32_t t = cbeg + it * 32 * ASM_W + sub * 32 + lane;
      bool act = t < cend;
      int32_t el[6];
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        el[a] = act ? esort[a * E + t] : 0;
        if (el[a] == i) act = false;  // near pair: the near kernel's
      }
      float ar[KB][6], ai[KB][6];
#pragma unroll
      for (int j = 0; j < KB; ++j)
#pragma unroll
        for (int a = 0; a < 6; ++a) ar[j][a] = ai[j][a] = 0.f;
      if (act) {
        const bool soft = bc[el[0]] != 0;
        float sr[KB], si[KB], ear[KB], eai[KB], ebr[KB], ebi[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) sr[j] = si[j] = ear[j] = eai[j] = ebr[j] = ebi[j] = 0.f;
        // the point's 64-byte record (colour-sorted, point-major: four 16-byte loads); the next
        // point's is loaded while this one is computed
        const float4* qp = qaos + ((int64_t)qlo * E + t) * 4;
        float4 v0 = qp[0], v1 = qp[1], v2 = qp[2], v3 = qp[3];
        cf kqn[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) kqn[j] = kq[((int64_t)min(k0 + j, nk - 1) * Q + qlo) * E + t];
        for (int qq = qlo; qq < qhi; ++qq) {
          const float q[P32COUNT] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y, v2.z, v2.w, v3.x};
          cf kqc[KB];
#pragma unroll
          for (int j = 0; j < KB; ++j) kqc[j] = kqn[j];
          if (qq + 1 < qhi) {
            const float4* qn = qaos + ((int64_t)(qq + 1) * E + t) * 4;
            v0 = qn[0]; v1 = qn[1]; v2 = qn[2]; v3 = qn[3];
#pragma unroll
            for (int j = 0; j < KB; ++j) kqn[j] = kq[((int64_t)min(k0 + j, nk - 1) * Q + qq + 1) * E + t];
          }
          // geometry, shared by the KB wavenumbers
          // float-float geometry with lazy tails (distance, 1/R, nu_i.r)
          const ff rx = ff_diff_lazy(ff{q[0], q[3]}, xi[0]);
          const ff ry = ff_diff_lazy(ff{q[1], q[4]}, xi[1]);
          const ff rz = ff_diff_lazy(ff{q[2], q[5]}, xi[2]);
          const ff R2 = ff_norm2_lazy(rx, ry, rz);
          float invR;
          const ff R = ff_sqrt_lazy(R2, invR);
          const ff nr = ff_dot3_lazy(nui, rx, ry, rz);
          float rnu;
          if (R2.hi > far_r2) {
            rnu = (rx.hi + rx.lo) * q[6] + (ry.hi + ry.lo) * q[7] + (rz.hi + rz.lo) * q[8];
          } else {
            const ff nq[3] = {ff{q[6], q[10]}, ff{q[7], q[11]}, ff{q[8], q[12]}};
            const ff d = ff_dot3_lazy(nq, rx, ry, rz);
            rnu = d.hi + d.lo;
          }
          const float nn = nui[0].hi * q[6] + nui[1].hi * q[7] + nui[2].hi * q[8];
          const float wj = q[P32W];
          // the weight rides on 1/R and on r.nu/R^3: G and dG/dnu below are w G and w dG/dnu
          const float wiR = wj * invR, wrn = wj * (rnu * invR * invR * invR);
          float sh[6];
#pragma unroll
          for (int a = 0; a < 6; ++a) sh[a] = shp[qq * 6 + a];
#pragma unroll
          for (int j = 0; j < KB; ++j) {
            float c, s;
            cis_ffprod(k[j], R, c, s);
            const float kR = k[j].hi * R.hi;
            const float Gr = c * wiR, Gi = s * wiR;
            const float dGr = (-c - s * kR) * wrn, dGi = (c * kR - s) * wrn;
            float cg, sg;
            cis_ffprod(k[j], nr, cg, sg);
            const float g = cg, f = kinv[j] != 0.f ? sg * kinv[j] : nr.hi, dg = -k[j].hi * sg * nn, df = cg * nn;
            ear[j] = __fmaf_rn(g, dGr, __fmaf_rn(-dg, Gr, ear[j]));
            eai[j] = __fmaf_rn(g, dGi, __fmaf_rn(-dg, Gi, eai[j]));
            ebr[j] = __fmaf_rn(f, dGr, __fmaf_rn(-df, Gr, ebr[j]));
            ebi[j] = __fmaf_rn(f, dGi, __fmaf_rn(-df, Gi, ebi[j]));
            // into A: dG (hard) or -G (soft); into b: G kq (hard) or -dG kq (soft)
            const float war = soft ? -Gr : dGr, wai = soft ? -Gi : dGi;
            const float wbr = soft ? -dGr : Gr, wbi = soft ? -dGi : Gi;
#pragma unroll
            for (int a = 0; a < 6; ++a) {
              ar[j][a] = __fmaf_rn(sh[a], war, ar[j][a]);
              ai[j][a] = __fmaf_rn(sh[a], wai, ai[j][a]);
            }
            const cf kqv = kqc[j];
            sr[j] = __fmaf_rn(wbr, kqv.re, __fmaf_rn(-wbi, kqv.im, sr[j]));
            si[j] = __fmaf_rn(wbr, kqv.im, __fmaf_rn(wbi, kqv.re, si[j]));
          }
        }
#pragma unroll
        for (int j = 0; j < KB; ++j) {
          S[j].ar.add(ear[j]); S[j].ai.add(eai[j]);
          S[j].br.add(ebr[j]); S[j].bi.add(ebi[j]);
          S[j].sr.add(sr[j]); S[j].si.add(si[j]);
        }
      }
      // scatter into the row: the quadrature halves one after the other
#pragma unroll
      for (int hh = 0; hh < QS; ++hh) {
        if (act && h == hh) {
#pragma unroll
          for (int j = 0; j < KB; ++j) {
            if (GROW && j >= nkb) break;  // no system behind a ragged group's last slots
            cf* row = row_of(j);
#pragma unroll
            for (int a = 0; a < 6; ++a) {
              row[el[a] - w0].re += ar[j][a];
              row[el[a] - w0].im += ai[j][a];
            }
          }
        }
        if (QS > 1) bar_named(1 + rw, 32 * WR);
      }
    }
    if (QS == 1) bar_named(1 + rw, 32 * WR);  // the row's warps finish the colour (rows <= 8: ids 1..8)
  }
  if constexpr (MODE == 2) {  // the window to A, then its accumulator is free for the next one
    bar_named(1 + rw, 32 * WR);
    const int ww = win_lo[w + 1] - w0;
    if (valid)
      for (int j = 0; j < nkb; ++j) {
        const cf* r = row_of(j);
        cf* Arow = A + ((int64_t)(k0 + j) * N + i) * lda + w0;
        for (int c2 = wr * 32 + lane; c2 < ww; c2 += 32 * WR) Arow[c2] = r[c2];
      }
    bar_named(1 + rw, 32 * WR);
  }
  }  // windows
  // reduce the compensated sums across the warp in FP64 (6 values per row and wavenumber)
#pragma unroll
  for (int j = 0; j < KB; ++j) {
    const ksum* v[6] = {&S[j].ar, &S[j].ai, &S[j].br, &S[j].bi, &S[j].sr, &S[j].si};
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      double x = (double)v[u]->s + (double)v[u]->c;
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) part[rw][wr][j][u] = x;
    }
  }
  __syncthreads();
  if (!valid) return;
  for (int j = 0; j < nkb; ++j) {
    if constexpr (MODE == 0) {
      const cf* row = row_of(j);
      cf* Arow = A + ((int64_t)(k0 + j) * N + i) * lda;
      for (int64_t c2 = wr * 32 + lane; c2 < N; c2 += 32 * WR) Arow[c2] = row[c2];
    }
    if (wr == 0 && lane < 6) {
      double x = 0.0;
      for (int w = 0; w < WR; ++w) x += part[rw][w][j][lane];
      rowsum[((int64_t)(k0 + j) * N + i) * 6 + lane] = x;
    }
  }
}

// One level of a warp's halving exchange: v[0 .. 2 HALF) per lane; the lane keeps the upper or
// lower half (by `upper`), adds its partner's (lane ^ o) copy of that half and stores it in
// v[0 .. HALF).
template <int HALF, class T>
__device__ __forceinline__ void halving_exchange(T* v, int o, bool upper) {
#pragma unroll
  for (int m = 0; m < HALF; ++m) {
    const T send = upper ? v[m] : v[m + HALF];
    const T keep = upper ? v[m + HALF] : v[m];
    v[m] = keep + __shfl_xor_sync(0xffffffffu, send, o);
  }
}

// Near pairs (element contains node i) and the diagonal terms; one warp per row.
__global__ void __launch_bounds__(128) k_asm32_near(
    const double* __restrict__ nodes, const double* __restrict__ normals, const uint8_t* __restrict__ bc,
    const int32_t* __restrict__ elems, int64_t N, int64_t E, int QN, const int* __restrict__ nnear_d,
    const float4* __restrict__ naos, const float* __restrict__ nshape, const int32_t* __restrict__ n2e_off,
    const int32_t* __restrict__ n2e, const double* __restrict__ kv, const cd* __restrict__ known,
    cf* __restrict__ A, int64_t lda, const double* __restrict__ rowsum, cd* __restrict__ b, TwoPi3 tp) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int kk = blockIdx.y;
  if (i >= N) return;
  const ff k = ff_from_double(kv[kk]);
  const float kinv = kinv32(kv[kk]);
  const cd* kn = known + (int64_t)kk * N;
  ff xi[3], nui[3];
  for (int d = 0; d < 3; ++d) {
    xi[d] = ff_from_double(nodes[3 * i + d]);
    nui[d] = ff_from_double(normals[3 * i + d]);
  }
  cf* Arow = A + ((int64_t)kk * N + i) * lda;
  // The regularisation sums per lane in compensated FP32 (they cancel against the bulk's) and the
  // nodal sums per lane in FP32 (a lane holds a few points of one element); across the warp the
  // nodal sums are reduced by halving exchanges, so that each of six lanes ends with one node's
  // four sums, and the right-hand side accumulates in float-float: the GB300's FP64 pipe is too
  // narrow for per-point FP64 arithmetic here (per element, six lanes split their node's known
  // value into float-float: two FP64 conversions and subtractions each).
  ksum sal_r, sal_i, sbe_r, sbe_i;
  ff bsr = {0.f, 0.f}, bsi = {0.f, 0.f};
  const int node = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
  for (int32_t t = n2e_off[i]; t < n2e_off[i + 1]; ++t) {
    const int32_t e = n2e[t] >> 3, a0 = n2e[t] & 7;
    const int np = nnear_d[a0];
    float hr[6], hi[6], gr[6], gi[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) { hr[a] = hi[a] = gr[a] = gi[a] = 0.f; }
    for (int qq = lane; qq < np; qq += 32) {
      const float4* qp = naos + (((int64_t)e * 6 + a0) * QN + qq) * 4;  // the point's 64-byte record
      const float4 v0 = qp[0], v1 = qp[1], v2 = qp[2], v3 = qp[3];
      const float q[P32COUNT] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y, v2.z, v2.w, v3.x};
      Kern32 K;
      kernel32(k, kinv, xi, nui, tp, q, K);
      const float wj = q[P32W];
      // w K enters exactly: the product's rounding error joins the compensation term
      auto add_exact = [&](ksum& acc, float x) {
        const float p = wj * x;
        acc.add(p);
        acc.c += __fmaf_rn(wj, x, -p);
      };
      add_exact(sal_r, K.alr); add_exact(sal_i, K.ali);
      add_exact(sbe_r, K.ber); add_exact(sbe_i, K.bei);
      const float* sh = nshape + ((int64_t)a0 * QN + qq) * 6;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const float cw = wj * sh[a];
        hr[a] = __fmaf_rn(cw, K.dGr, hr[a]); hi[a] = __fmaf_rn(cw, K.dGi, hi[a]);
        gr[a] = __fmaf_rn(cw, K.Gr, gr[a]);  gi[a] = __fmaf_rn(cw, K.Gi, gi[a]);
      }
    }
    // node a: u[4a .. 4a+3] = h re, h im, g re, g im; nodes 6, 7 are padding.  The first two
    // levels add partial sums of 2 and 4 lanes in FP32 (small against the total), the rest in
    // float-float (FP32 pipes: the FP64 pipe of the GB300 is too narrow for this reduction).
    float u[32];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      u[4 * a] = hr[a]; u[4 * a + 1] = hi[a]; u[4 * a + 2] = gr[a]; u[4 * a + 3] = gi[a];
    }
#pragma unroll
    for (int m = 24; m < 32; ++m) u[m] = 0.f;
    halving_exchange<16>(u, 16, (lane & 16) != 0);
    halving_exchange<8>(u, 8, (lane & 8) != 0);
    ff v[4];
    {
      const bool up = (lane & 4) != 0;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float send = up ? u[m] : u[m + 4], keep = up ? u[m + 4] : u[m];
        v[m] = ff_two_sum(keep, __shfl_xor_sync(0xffffffffu, send, 4));
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int o = 2; o > 0; o >>= 1) {
        const ff r = {__shfl_xor_sync(0xffffffffu, v[m].hi, o), __shfl_xor_sync(0xffffffffu, v[m].lo, o)};
        v[m] = ff_add(v[m], r);
      }
    if ((lane & 3) == 0 && node < 6) {  // this lane holds node `node`'s sums
      const int32_t j = elems[6 * (int64_t)e + node];
      const ff kr = ff_from_double(kn[j].re), ki = ff_from_double(kn[j].im);
      if (bc[j] == 0) {  // hard column: A += H, b += G known
        Arow[j].re += __fadd_rn(v[0].hi, v[0].lo); Arow[j].im += __fadd_rn(v[1].hi, v[1].lo);
        bsr = ff_add(bsr, ff_sub(ff_mul(v[2], kr), ff_mul(v[3], ki)));
        bsi = ff_add(bsi, ff_add(ff_mul(v[2], ki), ff_mul(v[3], kr)));
      } else {           // soft column: A -= G, b -= H known
        Arow[j].re -= __fadd_rn(v[2].hi, v[2].lo); Arow[j].im -= __fadd_rn(v[3].hi, v[3].lo);
        bsr = ff_sub(bsr, ff_sub(ff_mul(v[0], kr), ff_mul(v[1], ki)));
        bsi = ff_sub(bsi, ff_add(ff_mul(v[0], ki), ff_mul(v[1], kr)));
      }
    }
    __syncwarp();  // the next element (sharing nodes with this one) updates after these writes
  }
  for (int o = 16; o > 0; o >>= 1) {
    bsr = ff_add(bsr, ff{__shfl_xor_sync(0xffffffffu, bsr.hi, o), __shfl_xor_sync(0xffffffffu, bsr.lo, o)});
    bsi = ff_add(bsi, ff{__shfl_xor_sync(0xffffffffu, bsi.hi, o), __shfl_xor_sync(0xffffffffu, bsi.lo, o)});
  }
  double bs_r = ff_to_double(bsr), bs_i = ff_to_double(bsi);
  double al_r = sal_r.value(), al_i = sal_i.value(), be_r = sbe_r.value(), be_i = sbe_i.value();
  for (int o = 16; o > 0; o >>= 1) {
    al_r += __shfl_xor_sync(0xffffffffu, al_r, o); al_i += __shfl_xor_sync(0xffffffffu, al_i, o);
    be_r += __shfl_xor_sync(0xffffffffu, be_r, o); be_i += __shfl_xor_sync(0xffffffffu, be_i, o);
  }
  if (lane == 0) {
    const double* rs = rowsum + ((int64_t)kk * N + i) * 6;
    al_r += rs[0]; al_i += rs[1]; be_r += rs[2]; be_i += rs[3];
    bs_r += rs[4]; bs_i += rs[5];
    const cd ki = kn[i];
    const double fr = 4.0 * kPi + al_r, fi = al_i;
    if (bc[i] == 0) {
      Arow[i].re -= (float)fr; Arow[i].im -= (float)fi;
      bs_r += be_r * ki.re - be_i * ki.im; bs_i += be_r * ki.im + be_i * ki.re;
    } else {
      Arow[i].re -= (float)be_r; Arow[i].im -= (float)be_i;
      bs_r += fr * ki.re - fi * ki.im; bs_i += fr * ki.im + fi * ki.re;
    }
    b[(int64_t)kk * N + i] = {bs_r, bs_i};
  }
}

__global__ void k_known64(const double* __restrict__ nodes, const double* __restrict__ normals,
                          const uint8_t* __restrict__ bc, int64_t N, const double* __restrict__ kv, double dx,
                          double dy, double dz, cd* __restrict__ known);

static TwoPi3 two_pi3() {
  const double tp = 2.0 * kPi;
  TwoPi3 r;
  r.c1 = (float)tp;
  r.c2 = (float)(tp - (double)r.c1);
  // third term from the FP64 remainder refined by a long-double-free split of 2 pi's digits
  const double tail = 2.4492935982947064e-16;  // 2 pi - fl64(2 pi)
  r.c3 = (float)((tp - (double)r.c1 - (double)r.c2) + tail);
  r.inv = (float)(1.0 / tp);
  return r;
}

// Layout of c->qgeo32: standard points [P32COUNT][E*Q] (element-major, used by the field kernels),
// near points [P32COUNT][E*6*QN], the colour-sorted standard points [P32COUNT][Q][E], then the
// colour-sorted connectivity as int32 [6][E].
static float* sorted_table(bie_ctx* c) {
  const int64_t nq = c->E * c->rule.Q, nn = c->E * 6 * (int64_t)c->rule.QN;
  return c->qgeo32 + P32COUNT * (nq + nn);
}
static int32_t* sorted_elems(bie_ctx* c) {
  return reinterpret_cast<int32_t*>(sorted_table(c) + P32COUNT * c->E * c->rule.Q);
}
// the colour-sorted points again as 64-byte records [Q][E][16 floats], 16-byte aligned
static size_t sorted_aos_offset(bie_ctx* c) {
  const int64_t nq = c->E * c->rule.Q, nn = c->E * 6 * (int64_t)c->rule.QN;
  return ((size_t)(P32COUNT * (2 * nq + nn) + 6 * c->E) + 63) / 64 * 64;
}
static float4* sorted_aos(bie_ctx* c) { return reinterpret_cast<float4*>(c->qgeo32 + sorted_aos_offset(c)); }
// the near points as 64-byte records [E * 6 * QN][16 floats], after the sorted records
static float4* near_aos(bie_ctx* c) {
  return reinterpret_cast<float4*>(c->qgeo32 + sorted_aos_offset(c) + 16 * (size_t)c->E * c->rule.Q);
}
const float4* sorted_aos_ptr(bie_ctx* c) { return sorted_aos(c); }

const float* sorted_table_ptr(bie_ctx* c) { return sorted_table(c); }
const int32_t* sorted_elems_ptr(bie_ctx* c) { return sorted_elems(c); }

int ensure_mixed_tables(bie_ctx* c) {
  if (c->qgeo32) return BIE_OK;
  const int64_t nq = c->E * c->rule.Q, nn = c->E * 6 * (int64_t)c->rule.QN;
  BIE_TRY(dev_alloc(c, (void**)&c->qgeo32, (sorted_aos_offset(c) + 16 * (size_t)(nq + nn)) * sizeof(float)));
  BIE_LAUNCH(k_points_to32<<<(unsigned)((nq + 255) / 256), 256, 0, c->stream>>>(c->qgeo, nq, c->qgeo32, nullptr));
  BIE_LAUNCH(k_points_to32<<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(c->ngeo, nn, c->qgeo32 + P32COUNT * nq,
                                                                                near_aos(c)));
  BIE_LAUNCH(k_points_to32_sorted<<<(unsigned)((nq + 255) / 256), 256, 0, c->stream>>>(
      c->qgeo, c->elem_perm, c->elems, c->E, c->rule.Q, sorted_table(c), sorted_elems(c), sorted_aos(c)));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

// Assembles nk FP32 systems: A [nk][N][lda] (cf), b [nk][N] (cd).  known [nk][N] (cd) receives the
// known boundary values; rowsum scratch: nk * N * 6 doubles; kq scratch: nk * E * Q cf (the known
// values at the quadrature points, used by the uniform-condition bulk kernel; may be NULL).
// (3 x longest element edge)^2: beyond it a pair's r.nu is formed in FP32 (once per geometry)
double far_radius2(bie_ctx* c) {
  if (!(c->far_r2 > 0.0)) {
    double h2 = 0.0;
    for (int64_t e = 0; e < c->E; ++e)
      for (int a = 0; a < 3; ++a) {
        const int32_t p = c->h_elems[6 * e + a], q = c->h_elems[6 * e + (a + 1) % 3];
        double d2 = 0.0;
        for (int x = 0; x < 3; ++x) {
          const double d = c->h_nodes[3 * p + x] - c->h_nodes[3 * q + x];
          d2 += d * d;
        }
        h2 = std::max(h2, d2);
      }
    c->far_r2 = 9.0 * h2;
  }
  return c->far_r2;
}

int assemble32(bie_ctx* c, const double* kv, int nk, cf* A, int64_t lda, cd* b, cd* known, double* rowsum, cf* kq) {
  const int64_t N = c->N;
  BIE_TRY(ensure_mixed_tables(c));
  dim3 gk((unsigned)((N + 255) / 256), nk);
  BIE_LAUNCH(k_known64<<<gk, 256, 0, c->stream>>>(c->nodes, c->normals, c->bc, N, kv, c->dir[0], c->dir[1], c->dir[2], known));
  int rows = 16 / ASM_W;
  while (rows > 1 && (size_t)rows * N * sizeof(cf) > 200 * 1024) rows /= 2;
  const size_t smem = (size_t)rows * N * sizeof(cf);
  if (smem > 200 * 1024)
    return fail(BIE_ERR_INVALID_ARG, "N = " + std::to_string(N) + " too large for the FP32 shared-memory row accumulator");
  if (c->rule.Q > 64) return fail(BIE_ERR_INVALID_ARG, "standard rule too large");
  const TwoPi3 tp = two_pi3();
  far_radius2(c);
  if (c->uniform_bc < 0) {  // does every element carry one condition on its six nodes?
    c->uniform_bc = 1;
    for (int64_t e = 0; e < c->E && c->uniform_bc; ++e)
      for (int a = 1; a < 6; ++a)
        if (c->h_bc[c->h_elems[6 * e + a]] != c->h_bc[c->h_elems[6 * e]]) c->uniform_bc = 0;
  }
  // the uniform-condition kernel: KB = 2 wavenumbers per thread with the quadrature points of an
  // element split over two warps (2 rows x 4 warps, 256 threads); its rows in shared memory while
  // two CTAs fit an SM, else (large N) in A itself; KB = 1 (4 rows x 2 warps) on request
  int kb = (kq && c->uniform_bc == 1) ? c->asm_kb : 0;
  if (kb >= 1) {
    const int64_t E = c->E;
    dim3 gq((unsigned)((E + 255) / 256), nk);
    BIE_LAUNCH(k_known_q32<<<gq, 256, 0, c->stream>>>(sorted_elems(c), E, c->rule.Q, c->qshape32, known, N, kq));
    if (kb == 2) {
      const int urows = 2;
      const bool grow = (size_t)urows * 2 * N * sizeof(cf) > 100 * 1024;
      // large N: window by window in shared memory where the mesh has column windows
      // ("asm.windows" 0 keeps the rows in A)
      const bool win = grow && c->nwin > 1 && c->asm_windows != 0 &&
                       (size_t)urows * 2 * c->win_max * sizeof(cf) <= 100 * 1024;
      const size_t usmem = win ? (size_t)urows * 2 * c->win_max * sizeof(cf) : grow ? 0 : (size_t)urows * 2 * N * sizeof(cf);
      dim3 gu((unsigned)((N + urows - 1) / urows), (unsigned)((nk + 1) / 2));
      if (win) {
        BIE_TRY((set_smem_max(k_asm32_bulk_u<2, 2, 2>)));
        BIE_LAUNCH(k_asm32_bulk_u<2, 2, 2><<<gu, 32 * urows * ASM_W * 2, usmem, c->stream>>>(
            c->nodes, c->normals, c->bc, sorted_elems(c), N, E, c->rule.Q, sorted_aos(c), c->qshape32, c->color_off,
            c->ncolors, kv, nk, kq, A, lda, rowsum, urows, tp, (float)c->far_r2, c->win_lo, c->wcol_off, c->nwin,
            c->win_max));
      } else if (grow) {
        BIE_LAUNCH(k_asm32_bulk_u<2, 2, 1><<<gu, 32 * urows * ASM_W * 2, 0, c->stream>>>(
            c->nodes, c->normals, c->bc, sorted_elems(c), N, E, c->rule.Q, sorted_aos(c), c->qshape32, c->color_off,
            c->ncolors, kv, nk, kq, A, lda, rowsum, urows, tp, (float)c->far_r2, c->win_lo, c->wcol_off, c->nwin,
            c->win_max));
      } else {
        BIE_TRY((set_smem_max(k_asm32_bulk_u<2, 2, 0>)));
        BIE_LAUNCH(k_asm32_bulk_u<2, 2, 0><<<gu, 32 * urows * ASM_W * 2, usmem, c->stream>>>(
            c->nodes, c->normals, c->bc, sorted_elems(c), N, E, c->rule.Q, sorted_aos(c), c->qshape32, c->color_off,
            c->ncolors, kv, nk, kq, A, lda, rowsum, urows, tp, (float)c->far_r2, c->win_lo, c->wcol_off, c->nwin,
            c->win_max));
      }
    } else {
      int urows = 4;
      while (urows > 1 && (size_t)urows * N * sizeof(cf) > 200 * 1024) urows /= 2;
      const bool grow = (size_t)urows * N * sizeof(cf) > 200 * 1024;
      if (grow) urows = 4;
      const size_t usmem = grow ? 0 : (size_t)urows * N * sizeof(cf);
      dim3 gu((unsigned)((N + urows - 1) / urows), (unsigned)nk);
      if (grow) {
        BIE_LAUNCH(k_asm32_bulk_u<1, 1, 1><<<gu, 32 * urows * ASM_W, 0, c->stream>>>(
            c->nodes, c->normals, c->bc, sorted_elems(c), N, E, c->rule.Q, sorted_aos(c), c->qshape32, c->color_off,
            c->ncolors, kv, nk, kq, A, lda, rowsum, urows, tp, (float)c->far_r2, c->win_lo, c->wcol_off, c->nwin,
            c->win_max));
      } else {
        BIE_TRY((set_smem_max(k_asm32_bulk_u<1, 1, 0>)));
        BIE_LAUNCH(k_asm32_bulk_u<1, 1, 0><<<gu, 32 * urows * ASM_W, usmem, c->stream>>>(
            c->nodes, c->normals, c->bc, sorted_elems(c), N, E, c->rule.Q, sorted_aos(c), c->qshape32, c->color_off,
            c->ncolors, kv, nk, kq, A, lda, rowsum, urows, tp, (float)c->far_r2, c->win_lo, c->wcol_off, c->nwin,
            c->win_max));
      }
    }
  }
  if (kb == 0) {
    BIE_TRY((set_smem_max(k_asm32_bulk)));
    dim3 gb((unsigned)((N + rows - 1) / rows), nk);
    BIE_LAUNCH(k_asm32_bulk<<<gb, 32 * rows * ASM_W, smem, c->stream>>>(c->nodes, c->normals, c->bc, sorted_elems(c), N,
                                                                        c->E, c->rule.Q, sorted_table(c), c->qshape32,
                                                                        c->color_off, c->ncolors, kv, known, A, lda,
                                                                        rowsum, rows, tp, (float)c->far_r2));
  }
  BIE_CUDA_TRY(cudaGetLastError());
  dim3 gn((unsigned)((N * 32 + 127) / 128), nk);
  BIE_LAUNCH(k_asm32_near<<<gn, 128, 0, c->stream>>>(c->nodes, c->normals, c->bc, c->elems, N, c->E, c->rule.QN, c->d_nnear,
                                          near_aos(c), c->nshape32, c->n2e_off, c->n2e, kv, known, A, lda,
                                          rowsum, b, tp));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

}  // namespace bie
