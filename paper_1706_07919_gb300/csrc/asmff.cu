// asmff.cu -- float-float assembly of Eq. (BRIEF) for the wavenumbers that need the FP64 system
// (those flagged near an interior resonance, see mixed.cu): the bulk (row, element) pairs of
// asm64.cu computed with every quantity carried as an unevaluated sum of two floats (about 48
// significant bits) on the FP32 pipes, which on this GPU run ~70x faster than the FP64 pipe.
// Output is the FP64 system of asm64.cu (entries rounded to double from float-float); the pairs
// whose element contains the collocation node stay with k_asm64_near.
//
// e^{i phi} to ~1e-14: phi (float-float) is reduced by n pi/2 with pi/2 split into three floats
// whose first two products with n are exact, then sin and cos of the reduced v, |v| <= pi/4, by
// their Taylor series written from the series: the leading terms in float-float by Horner's rule
// and the terms below 4e-9 in FP32 (truncation after v^15 and v^16: < 1e-16).
#include "bie_common.cuh"

namespace bie {

__device__ __forceinline__ ff ffx_add_f(ff a, float b) {  // ff + float
  const ff s = ff_two_sum(a.hi, b);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ ff ffx_mul_f(ff a, float b) {  // ff * float
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return ff_fast_two_sum(p, e);
}
// acc += a * b (ff * ff), accumulated with a two-sum on the heads
__device__ __forceinline__ void ffx_mac(ff& acc, ff a, ff b) { acc = ff_add(acc, ff_mul(a, b)); }
// The same for the short sums of one element's quadrature points: the product's head is added to
// acc.hi error-free and its error terms, with the addition's, are gathered in acc.lo without
// renormalising (12 instructions instead of 18; over a few terms the unevaluated sum stays within
// a few units of acc.hi's last place of the exact one)
__device__ __forceinline__ void ffx_mac_lazy(ff& acc, ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  const ff t = ff_two_sum(acc.hi, p);
  acc = {t.hi, __fadd_rn(acc.lo, __fadd_rn(t.lo, e))};
}
__device__ __forceinline__ ff ffx_recip(ff a) {  // 1 / a by one Newton step on the FP32 reciprocal
  const float y = 1.0f / a.hi;
  const ff e = ff_sub(ff{1.0f, 0.0f}, ffx_mul_f(a, y));  // 1 - a y, small
  return ffx_add_f(ffx_mul_f(e, y), y);
}

struct FFConst {
  float p1, p2, p3;            // pi/2 = p1 + p2 + p3, p1 and p2 with 16 significant bits
  float two_over_pi;
  ff s3, s5, s7, s9;           // -1/3!, 1/5!, -1/7!, 1/9!
  float s11, s13, s15;         // -1/11!, 1/13!, -1/15!
  ff c2, c4, c6, c8;           // -1/2!, 1/4!, -1/6!, 1/8!
  float c10, c12, c14, c16;    // -1/10!, 1/12!, -1/14!, 1/16!
};

__device__ __forceinline__ void cis_ff(ff phi, const FFConst& K, ff& c, ff& s) {
  const float nm = __fadd_rn(__fmul_rn(phi.hi, K.two_over_pi), kRoundMagic);  // |phi 2/pi| < 2^22
  const float n = __fsub_rn(nm, kRoundMagic);
  const float h = __fmaf_rn(-n, K.p1, phi.hi);  // exact (n p1 exact, result within the ulp grid)
  ff u = ff_two_sum(h, -n * K.p2);              // n p2 exact
  u = ffx_add_f(u, __fmaf_rn(-n, K.p3, phi.lo));
  const ff z = ff_sqr(u);
  // sin u = u + u z S(z)
  const float ts = __fmaf_rn(z.hi, __fmaf_rn(z.hi, K.s15, K.s13), K.s11);  // -1/11! + z/13! - z^2/15!
  ff S = ffx_add_f(K.s9, z.hi * ts);
  S = ff_add(K.s7, ff_mul(z, S));
  S = ff_add(K.s5, ff_mul(z, S));
  S = ff_add(K.s3, ff_mul(z, S));
  const ff sv = ff_add(u, ff_mul(ff_mul(u, z), S));
  // cos u = 1 + z C(z)
  const float tc = __fmaf_rn(z.hi, __fmaf_rn(z.hi, __fmaf_rn(z.hi, K.c16, K.c14), K.c12), K.c10);
  ff C = ffx_add_f(K.c8, z.hi * tc);
  C = ff_add(K.c6, ff_mul(z, C));
  C = ff_add(K.c4, ff_mul(z, C));
  C = ff_add(K.c2, ff_mul(z, C));
  const ff cv = ffx_add_f(ff_mul(z, C), 1.0f);
  const int q = __float_as_int(nm) & 3;
  const ff a = (q & 1) ? sv : cv, b = (q & 1) ? cv : sv;
  c = (q == 1 || q == 2) ? ff_neg(a) : a;
  s = (q >= 2) ? ff_neg(b) : b;
}

// Same outputs and launch shape as k_asm32_bulk (rows per CTA x ASMF_W warps per row, colours
// separated by block barriers), with a float-float row accumulator [rows][N] in shared memory, or
// for large N (GROW) in the output rows of A themselves (each row belongs to one CTA; the elements
// of a colour share no node, so the row's warps never touch the same entry between barriers),
// converted to FP64 once the row is complete.  The scatter and the right-hand side's products with
// the known values (given as float-float) run on the FP32 pipes: no FP64 arithmetic per element.
// With QS = 2 the quadrature points of an element are split over two sets of ASMF_W warps (four
// warps per row), so that two rows fit one CTA of 256 threads and two CTAs an SM (16 warps); the
// halves add into the row one after the other (a barrier of the row's warps in between).
constexpr int ASMF_W = 2;
template <bool GROW, int QS>
__global__ void __launch_bounds__(256, 2) k_asmff_bulk(
    const double* __restrict__ nodes, const double* __restrict__ normals, const uint8_t* __restrict__ bc,
    const int32_t* __restrict__ esort, int64_t N, int64_t E, int Q,
    const float4* __restrict__ qaos /* colour-sorted float-float points, 64-byte records [Q][E] */,
    const double* __restrict__ qshape,
    const int32_t* __restrict__ color_off, int ncolors, const double* __restrict__ kv,
    const float4* __restrict__ knf /* [nk][N] known values as float-float: re hi, re lo, im hi, im lo */,
    cd* __restrict__ A, cd* __restrict__ rowsum /* [nk][N][3] */, int rows, FFConst K) {
  constexpr int WR = ASMF_W * QS;  // warps per row
  extern __shared__ float4 accf[];
  __shared__ ff shp[64 * 6];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rw = warp / WR, wr = warp % WR, sub = wr % ASMF_W, h = wr / ASMF_W;
  const int kk = blockIdx.y;
  if (kv[kk] < 0.0) return;  // an idle slot of a re-assembly round (stream-ordered solves)
  const ff k = ff_from_double(kv[kk]);
  const bool kzero = !(kv[kk] > 0.0);  // the zero-frequency term: f takes its limit nu_i.r
  const ff kinv = ff_from_double(kzero ? 0.0 : 1.0 / kv[kk]);
  for (int t = threadIdx.x; t < Q * 6; t += blockDim.x) shp[t] = ff_from_double(qshape[t]);
  const int64_t i = (int64_t)blockIdx.x * rows + rw;
  const bool valid = i < N;
  // the row accumulates in float-float (re hi, re lo, im hi, im lo: 16 bytes, the size of a cd
  // entry), in shared memory or (GROW) in the output row itself, converted to FP64 at the end
  float4* row;
  if constexpr (GROW) {
    row = reinterpret_cast<float4*>(A + ((int64_t)kk * N + (valid ? i : 0)) * N);
    if (valid)
      for (int64_t j = wr * 32 + lane; j < N; j += 32 * WR) row[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    for (int64_t t = threadIdx.x; t < (int64_t)rows * N; t += blockDim.x) accf[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    row = accf + (int64_t)rw * N;
  }
  __syncthreads();
  const float4* kn = knf + (int64_t)kk * N;
  ff xi[3], nui[3];
  for (int d = 0; d < 3; ++d) {
    xi[d] = ff_from_double(valid ? nodes[3 * i + d] : 0.0);
    nui[d] = ff_from_double(valid ? normals[3 * i + d] : 0.0);
  }
  const int qlo = h * Q / QS, qhi = (h + 1) * Q / QS;
  ff alr = {0, 0}, ali = {0, 0}, ber = {0, 0}, bei = {0, 0}, bsr = {0, 0}, bsi = {0, 0};
  for (int col = 0; col < ncolors; ++col) {
    const int32_t cbeg = color_off[col], cend = color_off[col + 1];
    // the same trip count for all warps of the row (the barriers below are the row's)
    const int iters = valid ? (cend - cbeg + 32 * ASMF_W - 1) / (32 * ASMF_W) : 0;
    for (int it = 0; it < iters; ++it) {
      const int32_t t = cbeg + it * 32 * ASMF_W + sub * 32 + lane;
      bool act = t < cend;
      int32_t el[6];
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        el[a] = act ? esort[a * E + t] : 0;
        if (el[a] == i) act = false;  // near pair: the near kernel's
      }
      ff hr[6], hi[6], gr[6], gi[6];
#pragma unroll
      for (int a = 0; a < 6; ++a) hr[a] = hi[a] = gr[a] = gi[a] = ff{0.f, 0.f};
      for (int qq = qlo; act && qq < qhi; ++qq) {
        const float4* qp = qaos + ((int64_t)qq * E + t) * 4;  // x hi, x lo, nu hi, w, nu lo, w lo
        const float4 v0 = qp[0], v1 = qp[1], v2 = qp[2], v3 = qp[3];
        const ff qx = {v0.x, v0.w}, qy = {v0.y, v1.x}, qz = {v0.z, v1.y};
        const ff nx = {v1.z, v2.z}, ny = {v1.w, v2.w}, nz = {v2.x, v3.x};
        const ff wj = {v2.y, v3.y};
        const ff rx = ff_sub(qx, xi[0]), ry = ff_sub(qy, xi[1]), rz = ff_sub(qz, xi[2]);
        const ff R = ff_sqrt(ff_add(ff_add(ff_sqr(rx), ff_sqr(ry)), ff_sqr(rz)));
        const ff invR = ffx_recip(R);
        const ff kR = ff_mul(k, R);
        ff c, s;
        cis_ff(kR, K, c, s);
        const ff Gr = ff_mul(c, invR), Gi = ff_mul(s, invR);
        const ff rnu = ff_add(ff_add(ff_mul(rx, nx), ff_mul(ry, ny)), ff_mul(rz, nz));
        const ff rn = ff_mul(rnu, ff_mul(invR, ff_sqr(invR)));
        // (c + i s)(i kR - 1) = (-c - s kR) + i (c kR - s)
        const ff dGr = ff_mul(ff_neg(ff_add(c, ff_mul(s, kR))), rn);
        const ff dGi = ff_mul(ff_sub(ff_mul(c, kR), s), rn);
        const ff nr = ff_add(ff_add(ff_mul(nui[0], rx), ff_mul(nui[1], ry)), ff_mul(nui[2], rz));
        ff cg, sg;
        cis_ff(ff_mul(k, nr), K, cg, sg);
        const ff nn = ff_add(ff_add(ff_mul(nui[0], nx), ff_mul(nui[1], ny)), ff_mul(nui[2], nz));
        const ff f = kzero ? nr : ff_mul(sg, kinv), dg = ff_neg(ff_mul(ff_mul(k, sg), nn)), df = ff_mul(cg, nn);
        // row sums: w J [g dG - dg G], w J [f dG - df G]
        ffx_mac(alr, wj, ff_sub(ff_mul(cg, dGr), ff_mul(dg, Gr)));
        ffx_mac(ali, wj, ff_sub(ff_mul(cg, dGi), ff_mul(dg, Gi)));
        ffx_mac(ber, wj, ff_sub(ff_mul(f, dGr), ff_mul(df, Gr)));
        ffx_mac(bei, wj, ff_sub(ff_mul(f, dGi), ff_mul(df, Gi)));
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          const ff cw = ff_mul(wj, shp[qq * 6 + a]);
          ffx_mac_lazy(hr[a], cw, dGr);
          ffx_mac_lazy(hi[a], cw, dGi);
          ffx_mac_lazy(gr[a], cw, Gr);
          ffx_mac_lazy(gi[a], cw, Gi);
        }
      }
#pragma unroll
      for (int hh = 0; hh < QS; ++hh) {  // the quadrature halves add into the row in turn
        if (act && h == hh) {
#pragma unroll
          for (int a = 0; a < 6; ++a) {
            const int32_t j = el[a];
            const float4 k4 = kn[j];
            const ff kr = {k4.x, k4.y}, ki = {k4.z, k4.w};
            // hard column: A += H, b += Gm P'_known; soft column: A -= Gm, b -= H P_known
            const bool hard = bc[j] == 0;
            const ff ar = hard ? hr[a] : ff_neg(gr[a]), ai = hard ? hi[a] : ff_neg(gi[a]);
            const ff br = hard ? gr[a] : ff_neg(hr[a]), bi = hard ? gi[a] : ff_neg(hi[a]);
            float4 v = row[j];
            const ff nr = ff_add(ff{v.x, v.y}, ar), ni = ff_add(ff{v.z, v.w}, ai);
            row[j] = make_float4(nr.hi, nr.lo, ni.hi, ni.lo);
            bsr = ff_add(bsr, ff_sub(ff_mul(br, kr), ff_mul(bi, ki)));
            bsi = ff_add(bsi, ff_add(ff_mul(br, ki), ff_mul(bi, kr)));
          }
        }
        if (QS > 1) bar_named(1 + rw, 32 * WR);
      }
    }
    if (QS == 1) bar_named(1 + rw, 32 * WR);  // the row's warps finish the colour (rows <= 8: ids 1..8)
  }
  // combine the lanes' and the row's warps' sums in FP64
  double v[6] = {ff_to_double(alr), ff_to_double(ali), ff_to_double(ber), ff_to_double(bei), ff_to_double(bsr),
                 ff_to_double(bsi)};
#pragma unroll
  for (int u = 0; u < 6; ++u)
    for (int o = 16; o > 0; o >>= 1) v[u] += __shfl_xor_sync(0xffffffffu, v[u], o);
  __shared__ double part[8][WR][6];
  if (lane == 0)
    for (int u = 0; u < 6; ++u) part[rw][wr][u] = v[u];
  __syncthreads();
  if (valid) {
    // the row to FP64: from shared memory, or (GROW) in place, each entry by the thread that reads it
    cd* Arow = A + ((int64_t)kk * N + i) * N;
    for (int64_t j = wr * 32 + lane; j < N; j += 32 * WR) {
      const float4 v = row[j];
      Arow[j] = {ff_to_double(ff{v.x, v.y}), ff_to_double(ff{v.z, v.w})};
    }
    if (wr == 0 && lane == 0) {
      double w[6] = {0, 0, 0, 0, 0, 0};
      for (int s2 = 0; s2 < WR; ++s2)
        for (int u = 0; u < 6; ++u) w[u] += part[rw][s2][u];
      cd* rs = rowsum + ((int64_t)kk * N + i) * 3;
      rs[0] = {w[0], w[1]};
      rs[1] = {w[2], w[3]};
      rs[2] = {w[4], w[5]};
    }
  }
}

static FFConst make_ffconst() {
  FFConst K;
  const double pio2 = 1.57079632679489661923132169163975144;
  auto round_bits = [](double x, int bits) {  // x rounded to `bits` significant bits
    int ex;
    const double m = std::frexp(x, &ex);
    return std::ldexp(std::nearbyint(std::ldexp(m, bits)), ex - bits);
  };
  const double p1 = round_bits(pio2, 16);
  const double p2 = round_bits(pio2 - p1, 16);
  K.p1 = (float)p1;
  K.p2 = (float)p2;
  K.p3 = (float)(pio2 - p1 - p2);
  K.two_over_pi = (float)(1.0 / pio2);
  double fact[17];
  fact[0] = 1.0;
  for (int n = 1; n <= 16; ++n) fact[n] = fact[n - 1] * n;
  auto sgn = [](int n) { return ((n / 2) % 2) ? -1.0 : 1.0; };  // sign of the x^n term of sin / cos
  K.s3 = ff_from_double(sgn(3) / fact[3]);
  K.s5 = ff_from_double(sgn(5) / fact[5]);
  K.s7 = ff_from_double(sgn(7) / fact[7]);
  K.s9 = ff_from_double(sgn(9) / fact[9]);
  K.s11 = (float)(sgn(11) / fact[11]);
  K.s13 = (float)(sgn(13) / fact[13]);
  K.s15 = (float)(sgn(15) / fact[15]);
  K.c2 = ff_from_double(sgn(2) / fact[2]);
  K.c4 = ff_from_double(sgn(4) / fact[4]);
  K.c6 = ff_from_double(sgn(6) / fact[6]);
  K.c8 = ff_from_double(sgn(8) / fact[8]);
  K.c10 = (float)(sgn(10) / fact[10]);
  K.c12 = (float)(sgn(12) / fact[12]);
  K.c14 = (float)(sgn(14) / fact[14]);
  K.c16 = (float)(sgn(16) / fact[16]);
  return K;
}

int ensure_mixed_tables(bie_ctx* c);
const float4* sorted_aos_ptr(bie_ctx* c);
const int32_t* sorted_elems_ptr(bie_ctx* c);

// known values [n] (FP64) split into float-float: re hi, re lo, im hi, im lo
__global__ void k_known_ff(const cd* __restrict__ known, int64_t n, float4* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const cd v = known[t];
  const ff r = ff_from_double(v.re), i = ff_from_double(v.im);
  out[t] = make_float4(r.hi, r.lo, i.hi, i.lo);
}

// Bulk part of the FP64 system in float-float (the replacement of k_asm64_bulk in assemble64).
int assemble_ff_bulk(bie_ctx* c, const double* kv, int nk, cd* A, const cd* known, cd* rowsum) {
  const int64_t N = c->N;
  BIE_TRY(ensure_mixed_tables(c));
  BIE_TRY(ensure_buf(c, c->work6, (size_t)nk * N * sizeof(float4)));
  float4* knf = (float4*)c->work6.p;
  BIE_LAUNCH(k_known_ff<<<(unsigned)((nk * N + 255) / 256), 256, 0, c->stream>>>(known, nk * N, knf));
  // 2 rows x 4 warps (quadrature halves) when two such CTAs fit an SM, else 4 rows x 2 warps
  // shrunk to fit shared memory, else (large N) the rows accumulate in A itself
  const bool split = (size_t)2 * N * sizeof(cd) <= 100 * 1024;
  int rows = split ? 2 : 4;
  while (!split && rows > 1 && (size_t)rows * N * sizeof(cd) > 200 * 1024) rows /= 2;
  const bool grow = (size_t)rows * N * sizeof(cd) > 200 * 1024;
  if (grow) rows = 4;
  const size_t smem = grow ? 0 : (size_t)rows * N * sizeof(cd);
  if (c->rule.Q > 64) return fail(BIE_ERR_INVALID_ARG, "standard rule too large");
  static const FFConst K = make_ffconst();
  dim3 gb((unsigned)((N + rows - 1) / rows), nk);
  if (grow) {
    BIE_LAUNCH(k_asmff_bulk<true, 1><<<gb, 32 * rows * ASMF_W, 0, c->stream>>>(
        c->nodes, c->normals, c->bc, sorted_elems_ptr(c), N, c->E, c->rule.Q, sorted_aos_ptr(c),
        c->qshape, c->color_off, c->ncolors, kv, knf, A, rowsum, rows, K));
  } else if (split) {
    BIE_TRY((set_smem_max(k_asmff_bulk<false, 2>)));
    BIE_LAUNCH(k_asmff_bulk<false, 2><<<gb, 32 * rows * ASMF_W * 2, smem, c->stream>>>(
        c->nodes, c->normals, c->bc, sorted_elems_ptr(c), N, c->E, c->rule.Q, sorted_aos_ptr(c),
        c->qshape, c->color_off, c->ncolors, kv, knf, A, rowsum, rows, K));
  } else {
    BIE_TRY((set_smem_max(k_asmff_bulk<false, 1>)));
    BIE_LAUNCH(k_asmff_bulk<false, 1><<<gb, 32 * rows * ASMF_W, smem, c->stream>>>(
        c->nodes, c->normals, c->bc, sorted_elems_ptr(c), N, c->E, c->rule.Q, sorted_aos_ptr(c),
        c->qshape, c->color_off, c->ncolors, kv, knf, A, rowsum, rows, K));
  }
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

}  // namespace bie
