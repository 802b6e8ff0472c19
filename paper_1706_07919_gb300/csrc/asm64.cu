// asm64.cu -- FP64 assembly of the boundary-regularised system Eq. (BRIEF) (Sec. 3, App. A, B).
//
// Row i (collocation node x_i, normal nu_i) of the scattered-field system:
//   sum_j [H_ij - (4 pi + alpha_i) d_ij] P_j - sum_j [Gm_ij + beta_i d_ij] P'_j = 0
// with H_ij = sum w J N_a dG(x_i, x)/dnu, Gm_ij = sum w J N_a G, alpha_i = sum w J [g dG - dg G],
// beta_i = sum w J [f dG - df G]; g = cos(k nu_i.(x - x_i)), f = sin(k nu_i.(x - x_i)) / k
// (Eqs. f_function, g_function) and the App. B term 4 pi P(x_i).  Hard columns keep P_j as the
// unknown, soft columns P'_j; the known boundary values (Sec. 4) go to the right-hand side.
//
// Work split: k_asm64_bulk does every (row, element) pair whose element does not contain the
// row's node (standard rule); one warp owns one row, its lanes take the elements of one colour at
// a time (elements of a colour share no node, so the shared-memory row accumulator needs no
// atomics).  k_asm64_near then adds the pairs whose element contains node i (near rule, collapsed
// on the node) and applies the diagonal terms.
#include "bie_common.cuh"

namespace bie {

// Known scattered-field boundary values for unit incident amplitude exp(i k d.x) (Sec. 4):
// hard node: dP/dnu = -i k (d.nu) exp(i k d.x); soft node: P = -exp(i k d.x).
__global__ void k_known64(const double* __restrict__ nodes, const double* __restrict__ normals,
                          const uint8_t* __restrict__ bc, int64_t N, const double* __restrict__ kv,
                          double dx, double dy, double dz, cd* __restrict__ known) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int kk = blockIdx.y;
  if (j >= N) return;
  double k = kv[kk];
  if (k < 0.0) return;  // an idle slot of a re-assembly round (stream-ordered solves)
  double ph = k * (dx * nodes[3 * j] + dy * nodes[3 * j + 1] + dz * nodes[3 * j + 2]);
  double s, c;
  sincos(ph, &s, &c);
  cd v;
  if (bc[j]) {
    v = {-c, -s};
  } else {
    double dn = dx * normals[3 * j] + dy * normals[3 * j + 1] + dz * normals[3 * j + 2];
    // -i k dn (c + i s) = k dn s - i k dn c
    v = {k * dn * s, -k * dn * c};
  }
  known[(int64_t)kk * N + j] = v;
}

struct Kern64 {
  cd G, dG;         // G(x_i, x) and dG/dnu(x)
  cd al, be;        // w J [g dG - dg G], w J [f dG - df G] (without w J)
};

// Kernel values of Eq. BRIEF at one quadrature point.
__device__ __forceinline__ void kernel64(double k, const double* xi, const double* nui, double x, double y,
                                         double z, double nx, double ny, double nz, Kern64& o) {
  double rx = x - xi[0], ry = y - xi[1], rz = z - xi[2];
  double R2 = rx * rx + ry * ry + rz * rz;
  double R = sqrt(R2);
  double invR = 1.0 / R;
  double kR = k * R;
  double s, c;
  sincos(kR, &s, &c);
  o.G = {c * invR, s * invR};
  double rn = (rx * nx + ry * ny + rz * nz) * invR * invR * invR;
  // (c + i s)(i kR - 1) = (-c - s kR) + i (c kR - s)
  o.dG = {(-c - s * kR) * rn, (c * kR - s) * rn};
  const double nr = nui[0] * rx + nui[1] * ry + nui[2] * rz;
  double sa = k * nr;
  double sg, cg;
  sincos(sa, &sg, &cg);
  double nn = nui[0] * nx + nui[1] * ny + nui[2] * nz;
  // f = sin(k nu_i.r)/k, and its limit nu_i.r at k = 0 (the zero-frequency term)
  double g = cg, f = k > 0.0 ? sg / k : nr, dg = -k * sg * nn, df = cg * nn;
  o.al = {g * o.dG.re - dg * o.G.re, g * o.dG.im - dg * o.G.im};
  o.be = {f * o.dG.re - df * o.G.re, f * o.dG.im - df * o.G.im};
}

// grid: (ceil(N / ROWS), nk); block: 32 * ROWS; dynamic smem: ROWS * N * sizeof(cd), or none
// with GROW (large N), where each warp accumulates straight into its row of A.
template <bool GROW>
__global__ void __launch_bounds__(512) k_asm64_bulk(
    const double* __restrict__ nodes, const double* __restrict__ normals, const uint8_t* __restrict__ bc,
    const int32_t* __restrict__ elems, int64_t N, int64_t E, int Q, const double* __restrict__ qgeo,
    const double* __restrict__ qshape, const int32_t* __restrict__ color_off, int ncolors,
    const int32_t* __restrict__ perm, const double* __restrict__ kv, const cd* __restrict__ known,
    cd* __restrict__ A, cd* __restrict__ rowsum /* [nk][N][3]: alpha, beta, b */, int rows) {
  extern __shared__ cd acc[];  // [rows][N]
  __shared__ double shp[64 * 6];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kk = blockIdx.y;
  const double k = kv[kk];
  if (k < 0.0) return;  // an idle slot of a re-assembly round (stream-ordered solves)
  for (int t = threadIdx.x; t < Q * 6; t += blockDim.x) shp[t] = qshape[t];
  const int64_t i = (int64_t)blockIdx.x * rows + warp;
  if constexpr (GROW) {
    if (i < N)
      for (int64_t j = lane; j < N; j += 32) A[((int64_t)kk * N + i) * N + j] = {0.0, 0.0};
  } else {
    for (int64_t t = threadIdx.x; t < (int64_t)rows * N; t += blockDim.x) acc[t] = {0.0, 0.0};
  }
  __syncthreads();
  if (i < N) {
    cd* row = GROW ? A + ((int64_t)kk * N + i) * N : acc + (int64_t)warp * N;
    const cd* kn = known + (int64_t)kk * N;
    const double xi[3] = {nodes[3 * i], nodes[3 * i + 1], nodes[3 * i + 2]};
    const double nui[3] = {normals[3 * i], normals[3 * i + 1], normals[3 * i + 2]};
    const int64_t EQ = E * Q;
    cd al = {0, 0}, be = {0, 0}, bsum = {0, 0};
    for (int col = 0; col < ncolors; ++col) {
      for (int32_t t = color_off[col] + lane; t < color_off[col + 1]; t += 32) {
        const int32_t e = perm[t];
        int32_t el[6];
        bool near = false;
        for (int a = 0; a < 6; ++a) {
          el[a] = elems[6 * (int64_t)e + a];
          near |= (el[a] == i);
        }
        if (near) continue;
        cd h[6], g[6];
        for (int a = 0; a < 6; ++a) { h[a] = {0, 0}; g[a] = {0, 0}; }
        for (int q = 0; q < Q; ++q) {
          const int64_t p = (int64_t)e * Q + q;
          Kern64 K;
          kernel64(k, xi, nui, qgeo[GX * EQ + p], qgeo[GY * EQ + p], qgeo[GZ * EQ + p], qgeo[GNX * EQ + p],
                   qgeo[GNY * EQ + p], qgeo[GNZ * EQ + p], K);
          const double wj = qgeo[GWJ * EQ + p];
          al.re += wj * K.al.re; al.im += wj * K.al.im;
          be.re += wj * K.be.re; be.im += wj * K.be.im;
          for (int a = 0; a < 6; ++a) {
            const double c = wj * shp[q * 6 + a];
            h[a].re += c * K.dG.re; h[a].im += c * K.dG.im;
            g[a].re += c * K.G.re;  g[a].im += c * K.G.im;
          }
        }
        for (int a = 0; a < 6; ++a) {
          const int32_t j = el[a];
          const cd kv_j = kn[j];
          if (bc[j] == 0) {  // hard column: A += H, b += Gm * P'_known
            row[j].re += h[a].re; row[j].im += h[a].im;
            bsum = cadd(bsum, cmul(g[a], kv_j));
          } else {           // soft column: A += -Gm, b += -H * P_known
            row[j].re -= g[a].re; row[j].im -= g[a].im;
            bsum = csub(bsum, cmul(h[a], kv_j));
          }
        }
      }
      __syncwarp();
    }
    // warp-reduce the row sums
    for (int o = 16; o > 0; o >>= 1) {
      al.re += __shfl_xor_sync(0xffffffffu, al.re, o); al.im += __shfl_xor_sync(0xffffffffu, al.im, o);
      be.re += __shfl_xor_sync(0xffffffffu, be.re, o); be.im += __shfl_xor_sync(0xffffffffu, be.im, o);
      bsum.re += __shfl_xor_sync(0xffffffffu, bsum.re, o); bsum.im += __shfl_xor_sync(0xffffffffu, bsum.im, o);
    }
    if constexpr (!GROW) {
      cd* Arow = A + ((int64_t)kk * N + i) * N;
      for (int64_t j = lane; j < N; j += 32) Arow[j] = row[j];
    }
    if (lane == 0) {
      cd* rs = rowsum + ((int64_t)kk * N + i) * 3;
      rs[0] = al; rs[1] = be; rs[2] = bsum;
    }
  }
}

// One warp per row i: the elements containing node i with the near rule of its local index,
// then the diagonal terms (App. B: 4 pi P(x_i); hard: -(4 pi + alpha_i) on A_ii, +beta_i P'_i on
// b_i; soft: -beta_i on A_ii, +(4 pi + alpha_i) P_i on b_i).
__global__ void __launch_bounds__(256) k_asm64_near(
    const double* __restrict__ nodes, const double* __restrict__ normals, const uint8_t* __restrict__ bc,
    const int32_t* __restrict__ elems, int64_t N, int64_t E, int QN, const int* __restrict__ nnear_d,
    const double* __restrict__ ngeo, const double* __restrict__ nshape, const int32_t* __restrict__ n2e_off,
    const int32_t* __restrict__ n2e, const double* __restrict__ kv, const cd* __restrict__ known,
    cd* __restrict__ A, const cd* __restrict__ rowsum, cd* __restrict__ b) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int kk = blockIdx.y;
  if (i >= N) return;
  const double k = kv[kk];
  if (k < 0.0) return;  // an idle slot of a re-assembly round (stream-ordered solves)
  const cd* kn = known + (int64_t)kk * N;
  const double xi[3] = {nodes[3 * i], nodes[3 * i + 1], nodes[3 * i + 2]};
  const double nui[3] = {normals[3 * i], normals[3 * i + 1], normals[3 * i + 2]};
  const int64_t tot = E * 6 * (int64_t)QN;
  cd* Arow = A + ((int64_t)kk * N + i) * N;
  cd al = {0, 0}, be = {0, 0}, bsum = {0, 0};
  for (int32_t t = n2e_off[i]; t < n2e_off[i + 1]; ++t) {
    const int32_t e = n2e[t] >> 3, a0 = n2e[t] & 7;
    const int np = nnear_d[a0];
    cd h[6], g[6];
    for (int a = 0; a < 6; ++a) { h[a] = {0, 0}; g[a] = {0, 0}; }
    for (int q = lane; q < np; q += 32) {
      const int64_t p = ((int64_t)e * 6 + a0) * QN + q;
      Kern64 K;
      kernel64(k, xi, nui, ngeo[GX * tot + p], ngeo[GY * tot + p], ngeo[GZ * tot + p], ngeo[GNX * tot + p],
               ngeo[GNY * tot + p], ngeo[GNZ * tot + p], K);
      const double wj = ngeo[GWJ * tot + p];
      al.re += wj * K.al.re; al.im += wj * K.al.im;
      be.re += wj * K.be.re; be.im += wj * K.be.im;
      const double* sh = nshape + ((int64_t)a0 * QN + q) * 6;
      for (int a = 0; a < 6; ++a) {
        const double c = wj * sh[a];
        h[a].re += c * K.dG.re; h[a].im += c * K.dG.im;
        g[a].re += c * K.G.re;  g[a].im += c * K.G.im;
      }
    }
    for (int a = 0; a < 6; ++a)
      for (int o = 16; o > 0; o >>= 1) {
        h[a].re += __shfl_xor_sync(0xffffffffu, h[a].re, o); h[a].im += __shfl_xor_sync(0xffffffffu, h[a].im, o);
        g[a].re += __shfl_xor_sync(0xffffffffu, g[a].re, o); g[a].im += __shfl_xor_sync(0xffffffffu, g[a].im, o);
      }
    if (lane == 0) {
      const int32_t* el = elems + 6 * (int64_t)e;
      for (int a = 0; a < 6; ++a) {
        const int32_t j = el[a];
        if (bc[j] == 0) {
          Arow[j].re += h[a].re; Arow[j].im += h[a].im;
          bsum = cadd(bsum, cmul(g[a], kn[j]));
        } else {
          Arow[j].re -= g[a].re; Arow[j].im -= g[a].im;
          bsum = csub(bsum, cmul(h[a], kn[j]));
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    al.re += __shfl_xor_sync(0xffffffffu, al.re, o); al.im += __shfl_xor_sync(0xffffffffu, al.im, o);
    be.re += __shfl_xor_sync(0xffffffffu, be.re, o); be.im += __shfl_xor_sync(0xffffffffu, be.im, o);
  }
  if (lane == 0) {
    const cd* rs = rowsum + ((int64_t)kk * N + i) * 3;
    al = cadd(al, rs[0]);
    be = cadd(be, rs[1]);
    bsum = cadd(bsum, rs[2]);
    const cd kv_i = kn[i];
    const cd fourpi_al = {4.0 * kPi + al.re, al.im};
    if (bc[i] == 0) {
      Arow[i] = csub(Arow[i], fourpi_al);
      bsum = cadd(bsum, cmul(be, kv_i));
    } else {
      Arow[i] = csub(Arow[i], be);
      bsum = cadd(bsum, cmul(fourpi_al, kv_i));
    }
    b[(int64_t)kk * N + i] = bsum;
  }
}

int assemble_ff_bulk(bie_ctx* c, const double* kv, int nk, cd* A, const cd* known, cd* rowsum);

// Assembles nk systems (FP64) for the device wavenumbers kv[0..nk): A [nk][N][N], b [nk][N].
// scratch: >= nk * N * (sizeof(cd) * 4) bytes.  ff_bulk: the bulk pairs in float-float on the
// FP32 pipes (asmff.cu) instead of FP64; the near pairs and the diagonal are FP64 either way.
int assemble64(bie_ctx* c, const double* kv, int nk, cd* A, cd* b, void* scratch, bool ff_bulk) {
  const int64_t N = c->N;
  cd* known = (cd*)scratch;
  cd* rowsum = known + (int64_t)nk * N;
  dim3 gk((unsigned)((N + 255) / 256), nk);
  BIE_LAUNCH(k_known64<<<gk, 256, 0, c->stream>>>(c->nodes, c->normals, c->bc, N, kv, c->dir[0], c->dir[1], c->dir[2], known));
  if (ff_bulk) {
    BIE_TRY(assemble_ff_bulk(c, kv, nk, A, known, rowsum));
  } else {
  int rows = 16;
  while (rows > 1 && (size_t)rows * N * sizeof(cd) > 200 * 1024) rows /= 2;
  const bool grow = (size_t)rows * N * sizeof(cd) > 200 * 1024;
  if (grow) rows = 8;
  size_t smem = grow ? 0 : (size_t)rows * N * sizeof(cd);
  if (c->rule.Q > 64) return fail(BIE_ERR_INVALID_ARG, "standard rule too large");
  dim3 gb((unsigned)((N + rows - 1) / rows), nk);
  if (grow) {
    BIE_LAUNCH(k_asm64_bulk<true><<<gb, 32 * rows, 0, c->stream>>>(c->nodes, c->normals, c->bc, c->elems, N, c->E,
                                                                   c->rule.Q, c->qgeo, c->qshape, c->color_off,
                                                                   c->ncolors, c->elem_perm, kv, known, A, rowsum,
                                                                   rows));
  } else {
    BIE_TRY((set_smem_max(k_asm64_bulk<false>)));
    BIE_LAUNCH(k_asm64_bulk<false><<<gb, 32 * rows, smem, c->stream>>>(c->nodes, c->normals, c->bc, c->elems, N,
                                                                       c->E, c->rule.Q, c->qgeo, c->qshape,
                                                                       c->color_off, c->ncolors, c->elem_perm, kv,
                                                                       known, A, rowsum, rows));
  }
  BIE_CUDA_TRY(cudaGetLastError());
  }
  dim3 gn((unsigned)((N * 32 + 255) / 256), nk);
  BIE_LAUNCH(k_asm64_near<<<gn, 256, 0, c->stream>>>(c->nodes, c->normals, c->bc, c->elems, N, c->E, c->rule.QN, c->d_nnear,
                                          c->ngeo, c->nshape, c->n2e_off, c->n2e, kv, known, A, rowsum, b));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

}  // namespace bie
