// mlp.cu -- the learned warm start of the frequency sweep: a 4-layer tanh perceptron that maps a
// node's features at wavenumber k to the (demodulated) surface unknown there, trained on the
// solutions of the directly solved wavenumbers and evaluated for the others as the initial guess
// of the Krylov solve (gmres.cu).  The warm start is not part of the paper's method (Sec. 4
// solves every frequency directly); it only changes where the iteration starts.
//
// Network (row-major weights, out x in):  h1 = tanh(W1 phi + b1)  (256 x 64),
//   h2 = tanh(W2 h1 + b2), h3 = tanh(W3 h2 + b3)  (256 x 256),  y = W4 h3 + b4  (2 x 256).
// Feature map phi (64 values) of node x with normal nu at wavenumber k: (x - c)/s, nu, k/kmax,
// (k/kmax)^2, and cos/sin of k * sc_q * (b_j . (x - c)) for 7 directions b_j (incidence d, the
// axes, the three face diagonals) and 4 scales sc_q = 0.5, 1, 1.5, 2.
// Loss (1/B) sum |y - t|^2, Adam with a cosine-decayed step size.
//
// The three hidden layers and their backward products are dense contractions and run on the
// tensor cores: tcgen05.mma kind::f16 with BF16 operands staged by TMA (128-byte swizzle) and
// FP32 accumulators in tensor memory, one 128 x N tile per CTA (N = 256, or 64 for dW1), with
// the activation, its derivative, the transposed copies the next GEMM needs, or the gradient
// accumulation fused into the epilogue.  The 2-wide output layer, the loss, the gather of a
// minibatch and the optimiser step run on the CUDA cores.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "tcgen05.cuh"

namespace bie {

using bf16 = __nv_bfloat16;

namespace mlp {

constexpr int D_IN = 64, W_H = 256, D_OUT = 2;
constexpr int64_t OFF_W1 = 0;
constexpr int64_t OFF_B1 = OFF_W1 + W_H * D_IN;
constexpr int64_t OFF_W2 = OFF_B1 + W_H;
constexpr int64_t OFF_B2 = OFF_W2 + W_H * W_H;
constexpr int64_t OFF_W3 = OFF_B2 + W_H;
constexpr int64_t OFF_B3 = OFF_W3 + W_H * W_H;
constexpr int64_t OFF_W4 = OFF_B3 + W_H;
constexpr int64_t OFF_B4 = OFF_W4 + D_OUT * W_H;
constexpr int64_t NPARAM = OFF_B4 + D_OUT;
static_assert(NPARAM == BIE_MLP_PARAMS, "parameter layout");

// ---------------------------------------------------------------------------------------------
// GEMM C[M][N] = sum_k A[M][K] B[N][K] (both K-major BF16), FP32 accumulation in TMEM.
// grid (ceil(M/128), kslices); CTA 128 threads; thread 0 issues the TMA loads (4-stage ring of
// 64-wide K chunks) and the MMAs (M = 128, N = NT, K = 16); all four warps run the epilogue on
// their 32 TMEM lanes.  Every wait is bounded and raises a flag in *err instead of hanging.
// ---------------------------------------------------------------------------------------------
constexpr int BM = 128, KC = 64, STAGES = 4, A_ST = BM * KC * 2;
enum { EPI_FWD = 0, EPI_BWD = 1, EPI_WGRAD = 2 };

struct Epi {
  const float* bias;   // FWD: [N]
  const bf16* hsave;   // BWD: [M][N] activation of this layer's input side
  bf16* out;           // FWD / BWD: [M][N] (optional)
  bf16* outT;          // FWD / BWD: [N][ldT] (optional)
  int64_t ldT;
  float* wgrad;        // WGRAD: [M][N] accumulated
};

template <int NT>
constexpr int gemm_smem_bytes() {
  return STAGES * (A_ST + NT * KC * 2) + 1024;
}

template <int NT, int EPI>
__global__ void __launch_bounds__(128, 1) k_gemm(const __grid_constant__ CUtensorMap tmA,
                                                 const __grid_constant__ CUtensorMap tmB, int M, int kc_per_cta,
                                                 int kc_total, Epi ep, int32_t* __restrict__ err) {
  constexpr int B_ST = NT * KC * 2;
  constexpr uint32_t TCOLS = NT;  // 64 or 256: powers of two >= 32
  extern __shared__ unsigned char smraw[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], accb;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_abort;
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  const uint32_t sA = tcx::smem_u32(sm), sB = sA + STAGES * A_ST;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * BM;
  const int kb = blockIdx.y * kc_per_cta;
  const int nch = min(kc_total, kb + kc_per_cta) - kb;
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tcx::mbar_init(tcx::smem_u32(&full[s]), 1);
      tcx::mbar_init(tcx::smem_u32(&empty[s]), 1);
    }
    tcx::mbar_init(tcx::smem_u32(&accb), 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) tcx::tmem_alloc(&tslot, TCOLS);
  tcx::fence_before();
  __syncthreads();
  tcx::fence_after();
  const uint32_t tmem = tslot;

  if (tid == 0) {
    auto load = [&](int c) {
      const int s = c % STAGES;
      const uint32_t fb = tcx::smem_u32(&full[s]);
      tcx::mbar_expect_tx(fb, A_ST + B_ST);
      tcx::tma_load_2d(sA + s * A_ST, &tmA, (kb + c) * KC, m0, fb);
      tcx::tma_load_2d(sB + s * B_ST, &tmB, (kb + c) * KC, 0, fb);
    };
    bool ok = nch > 0;
    int issued = 0, consumed = 0;
    for (int c = 0; c < min(STAGES, nch); ++c, ++issued) load(c);
    const uint32_t idesc = tcx::idesc_bf16(BM, NT);
    for (int c = 0; c < nch && ok; ++c) {
      const int s = c % STAGES;
      if (!tcx::mbar_wait(tcx::smem_u32(&full[s]), (c / STAGES) & 1, err, 1)) { ok = false; break; }
      consumed = c + 1;
      tcx::fence_after();
#pragma unroll
      for (int k = 0; k < KC / 16; ++k)
        tcx::mma_bf16(tmem, tcx::desc_sw128(sA + s * A_ST + k * 32), tcx::desc_sw128(sB + s * B_ST + k * 32), idesc,
                      (c | k) ? 1u : 0u);
      tcx::mma_commit(tcx::smem_u32(&empty[s]));
      // refill the previous chunk's slot once its MMAs are done (this chunk's MMAs stay queued)
      if (c >= 1 && c - 1 + STAGES < nch) {
        const int sp = (c - 1) % STAGES;
        if (!tcx::mbar_wait(tcx::smem_u32(&empty[sp]), ((c - 1) / STAGES) & 1, err, 2)) { ok = false; break; }
        load(c - 1 + STAGES);
        ++issued;
      }
    }
    if (ok) {
      tcx::mma_commit(tcx::smem_u32(&accb));
    } else {
      // let the copies still in flight land before the CTA's shared memory is released
      for (int c = consumed; c < issued; ++c)
        tcx::mbar_wait(tcx::smem_u32(&full[c % STAGES]), (c / STAGES) & 1, err, 4);
      s_abort = 1;
    }
  }
  // epilogue: wait for the accumulator (bounded; thread 0 may have given up)
  bool ok = false;
  for (uint32_t i = 0; i < (1u << 22); ++i) {
    if (tcx::mbar_try_wait(tcx::smem_u32(&accb), 0)) { ok = true; break; }
    if (s_abort) break;
  }
  if (!ok && lane == 0) atomicOr(err, 8);
  ok = __all_sync(0xffffffffu, ok);
  tcx::fence_after();
  if (ok) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < NT; c0 += 32) {
      float v[32];
      tcx::tmem_ld32(trow + c0, v);
      if (row >= M) continue;
      if constexpr (EPI == EPI_WGRAD) {
        float4* dst = reinterpret_cast<float4*>(ep.wgrad + (int64_t)row * NT + c0);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          atomicAdd(dst + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
      } else {
        __align__(16) bf16 o[32];
        if constexpr (EPI == EPI_FWD) {
#pragma unroll
          for (int j = 0; j < 32; ++j) o[j] = __float2bfloat16_rn(tanhf(v[j] + ep.bias[c0 + j]));
        } else {
          __align__(16) bf16 h[32];
          const uint4* hs = reinterpret_cast<const uint4*>(ep.hsave + (int64_t)row * NT + c0);
#pragma unroll
          for (int q = 0; q < 4; ++q) reinterpret_cast<uint4*>(h)[q] = hs[q];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float hv = __bfloat162float(h[j]);
            o[j] = __float2bfloat16_rn(v[j] * (1.0f - hv * hv));
          }
        }
        if (ep.out) {
          uint4* dst = reinterpret_cast<uint4*>(ep.out + (int64_t)row * NT + c0);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<const uint4*>(o)[q];
        }
        if (ep.outT) {
#pragma unroll
          for (int j = 0; j < 32; ++j) ep.outT[(int64_t)(c0 + j) * ep.ldT + row] = o[j];
        }
      }
    }
  }
  tcx::fence_before();
  __syncthreads();
  if (warp == 0) tcx::tmem_dealloc(tmem, TCOLS);
}

// ---------------------------------------------------------------------------------------------
// Output layer, loss and the first backward step (CUDA cores).  CTA = 8 warps, 32 rows; a warp
// takes 4 rows, a lane 8 consecutive hidden units.  Rows in [M, Mp) are padding: zero dZ3.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_head_train(const bf16* __restrict__ H3, int M, int Mp,
                                                    const float* __restrict__ theta, const float* __restrict__ T,
                                                    float inv_B, float* __restrict__ grad, bf16* __restrict__ dZ3,
                                                    bf16* __restrict__ dZ3T, int64_t ldT, float* __restrict__ loss) {
  __shared__ float w4[2][W_H];
  __shared__ float gw4[2][W_H], gb3[W_H], gb4[2], sl;
  __shared__ bf16 tile[32][W_H + 8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 2 * W_H; i += 256) {
    w4[i / W_H][i % W_H] = theta[OFF_W4 + i];
    gw4[i / W_H][i % W_H] = 0.f;
  }
  for (int i = tid; i < W_H; i += 256) gb3[i] = 0.f;
  if (tid < 2) gb4[tid] = 0.f;
  if (tid == 0) sl = 0.f;
  __syncthreads();
  const float b40 = theta[OFF_B4], b41 = theta[OFF_B4 + 1];
  const int c = lane * 8;
  float aw0[8], aw1[8], ab3[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) aw0[j] = aw1[j] = ab3[j] = 0.f;
  float ab40 = 0.f, ab41 = 0.f, al = 0.f;
  for (int u = 0; u < 4; ++u) {
    const int rl = warp * 4 + u, row = blockIdx.x * 32 + rl;
    __align__(16) bf16 hb[8];
    float h[8];
    if (row < M) *reinterpret_cast<uint4*>(hb) = *reinterpret_cast<const uint4*>(H3 + (int64_t)row * W_H + c);
    else *reinterpret_cast<uint4*>(hb) = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = __bfloat162float(hb[j]);
    float y0 = 0.f, y1 = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      y0 = fmaf(w4[0][c + j], h[j], y0);
      y1 = fmaf(w4[1][c + j], h[j], y1);
    }
    for (int o = 16; o > 0; o >>= 1) {
      y0 += __shfl_xor_sync(0xffffffffu, y0, o);
      y1 += __shfl_xor_sync(0xffffffffu, y1, o);
    }
    float dy0 = 0.f, dy1 = 0.f;
    if (row < M) {
      const float e0 = y0 + b40 - T[2 * (int64_t)row], e1 = y1 + b41 - T[2 * (int64_t)row + 1];
      if (lane == 0) al += (e0 * e0 + e1 * e1) * inv_B;
      dy0 = 2.f * e0 * inv_B;
      dy1 = 2.f * e1 * inv_B;
    }
    __align__(16) bf16 dz[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float d = (w4[0][c + j] * dy0 + w4[1][c + j] * dy1) * (1.f - h[j] * h[j]);
      aw0[j] = fmaf(dy0, h[j], aw0[j]);
      aw1[j] = fmaf(dy1, h[j], aw1[j]);
      ab3[j] += d;
      dz[j] = __float2bfloat16_rn(d);
      tile[rl][c + j] = dz[j];
    }
    if (lane == 0) { ab40 += dy0; ab41 += dy1; }
    if (row < Mp) *reinterpret_cast<uint4*>(dZ3 + (int64_t)row * W_H + c) = *reinterpret_cast<const uint4*>(dz);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    atomicAdd(&gw4[0][c + j], aw0[j]);
    atomicAdd(&gw4[1][c + j], aw1[j]);
    atomicAdd(&gb3[c + j], ab3[j]);
  }
  if (lane == 0) {
    atomicAdd(&gb4[0], ab40);
    atomicAdd(&gb4[1], ab41);
    atomicAdd(&sl, al);
  }
  __syncthreads();
  for (int i = tid; i < 2 * W_H; i += 256) atomicAdd(grad + OFF_W4 + i, gw4[i / W_H][i % W_H]);
  for (int i = tid; i < W_H; i += 256) atomicAdd(grad + OFF_B3 + i, gb3[i]);
  if (tid < 2) atomicAdd(grad + OFF_B4 + tid, gb4[tid]);
  if (tid == 0) atomicAdd(loss, sl);
  // transposed copy of dZ3: 32 consecutive rows per hidden unit
  const int r0 = blockIdx.x * 32;
  for (int i = tid; i < W_H * 32; i += 256) {
    const int cc = i >> 5, rr = i & 31;
    if (r0 + rr < Mp) dZ3T[(int64_t)cc * ldT + r0 + rr] = tile[rr][cc];
  }
}

// Column sums of dZ (rows of dZ^T) -> bias gradients of layers 1 and 2.  One warp per unit.
__global__ void k_bias_grad(const bf16* __restrict__ dZ1T, const bf16* __restrict__ dZ2T, int64_t ldT, int B,
                            float* __restrict__ grad) {
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w >= 2 * W_H) return;
  const bf16* row = (w < W_H ? dZ1T : dZ2T) + (int64_t)(w % W_H) * ldT;
  float s = 0.f;
  for (int i = lane; i < B; i += 32) s += __bfloat162float(row[i]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) grad[(w < W_H ? OFF_B1 : OFF_B2) + (w % W_H)] = s;
}

// ---- minibatch staging -----------------------------------------------------------------------
// X0[r] = X[idx[r]] (or X[r] when idx is null), X0T its transpose, Tb[r] = T[idx[r]]; rows
// r in [B, Bp) are zero.  CTA = 256 threads, 32 rows.  Block 0 advances the optimiser step.
__global__ void __launch_bounds__(256) k_gather(const bf16* __restrict__ X, const float* __restrict__ T,
                                                const int32_t* __restrict__ idx, int B, int Bp,
                                                bf16* __restrict__ X0, bf16* __restrict__ X0T,
                                                float* __restrict__ Tb, int64_t* step) {
  __shared__ bf16 tile[32][D_IN + 8];
  const int tid = threadIdx.x, r0 = blockIdx.x * 32;
  if (step && blockIdx.x == 0 && tid == 0) *step += 1;
  {
    const int rr = tid >> 3, q = tid & 7;  // 8 threads x 16 bytes per row
    const int r = r0 + rr;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (r < B) {
      const int64_t src = idx ? (int64_t)idx[r] : (int64_t)r;
      v = reinterpret_cast<const uint4*>(X + src * D_IN)[q];
      if (q < 2) Tb[2 * (int64_t)r + q] = T[2 * src + q];
    } else if (r < Bp && q < 2) {
      Tb[2 * (int64_t)r + q] = 0.f;
    }
    if (r < Bp) reinterpret_cast<uint4*>(X0 + (int64_t)r * D_IN)[q] = v;
    *reinterpret_cast<uint4*>(&tile[rr][q * 8]) = v;
  }
  __syncthreads();
  for (int i = tid; i < D_IN * 32; i += 256) {
    const int f = i >> 5, rr = i & 31;
    if (r0 + rr < Bp) X0T[(int64_t)f * Bp + r0 + rr] = tile[rr][f];
  }
}

__global__ void k_f32_to_bf16(const float* __restrict__ x, int64_t n, bf16* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}
__global__ void k_bf16_to_f32(const bf16* __restrict__ x, int64_t n, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __bfloat162float(x[i]);
}

// ---- optimiser --------------------------------------------------------------------------------
// Adam (Kingma & Ba, 2015) on the FP32 master copy with bias correction; the step size follows a
// cosine from lr to lr_min over `total` steps (constant when total = 0).  Writes the BF16
// operand copies (W1..W3 and the transposes of W2, W3) and clears the gradient.
__global__ void k_adam(float* __restrict__ theta, float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, const int64_t* __restrict__ step, float lr, float lr_min, int64_t total,
                       float b1, float b2, float eps, bf16* __restrict__ w1, bf16* __restrict__ w2,
                       bf16* __restrict__ w3, bf16* __restrict__ w2t, bf16* __restrict__ w3t) {
  const int64_t t = *step;
  float lr_t = lr;
  if (total > 0) {
    const double f = (double)min(t, total) / (double)total;
    lr_t = (float)(lr_min + 0.5 * (lr - lr_min) * (1.0 + cos(kPi * f)));
  }
  const float c1 = (float)(1.0 - pow((double)b1, (double)t)), c2 = (float)(1.0 - pow((double)b2, (double)t));
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < NPARAM; p += (int64_t)gridDim.x * blockDim.x) {
    const float g = grad[p];
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float th = theta[p] - lr_t * (mm / c1) / (sqrtf(vv / c2) + eps);
    theta[p] = th;
    grad[p] = 0.f;
    const bf16 hb = __float2bfloat16_rn(th);
    if (p < OFF_B1) {
      w1[p] = hb;
    } else if (p >= OFF_W2 && p < OFF_B2) {
      const int64_t q = p - OFF_W2;
      w2[q] = hb;
      w2t[(q % W_H) * W_H + q / W_H] = hb;
    } else if (p >= OFF_W3 && p < OFF_B3) {
      const int64_t q = p - OFF_W3;
      w3[q] = hb;
      w3t[(q % W_H) * W_H + q / W_H] = hb;
    }
  }
}

// BF16 operand copies from the master parameters (after they were set from the host).
__global__ void k_sync_weights(const float* __restrict__ theta, bf16* __restrict__ w1, bf16* __restrict__ w2,
                               bf16* __restrict__ w3, bf16* __restrict__ w2t, bf16* __restrict__ w3t) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < OFF_W4; p += (int64_t)gridDim.x * blockDim.x) {
    const bf16 hb = __float2bfloat16_rn(theta[p]);
    if (p < OFF_B1) {
      w1[p] = hb;
    } else if (p >= OFF_W2 && p < OFF_B2) {
      const int64_t q = p - OFF_W2;
      w2[q] = hb;
      w2t[(q % W_H) * W_H + q / W_H] = hb;
    } else if (p >= OFF_W3 && p < OFF_B3) {
      const int64_t q = p - OFF_W3;
      w3[q] = hb;
      w3t[(q % W_H) * W_H + q / W_H] = hb;
    }
  }
}

// ---- feature map and targets -------------------------------------------------------------------
// One thread per (wavenumber, node) row; phases reduced to [-pi, pi] in FP64, cos/sin in FP32.
__global__ void k_features(const double* __restrict__ nodes, const double* __restrict__ normals, int64_t N,
                           const double* __restrict__ kv, int nk, double dx, double dy, double dz, double cx,
                           double cy, double cz, double inv_scale, double inv_kmax, bf16* __restrict__ X,
                           float* __restrict__ Xf) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= (int64_t)nk * N) return;
  const int64_t i = row % N;
  const double k = kv[row / N];
  const double rx = nodes[3 * i] - cx, ry = nodes[3 * i + 1] - cy, rz = nodes[3 * i + 2] - cz;
  const double s2 = 0.70710678118654752440;
  const double proj[7] = {dx * rx + dy * ry + dz * rz, rx, ry, rz, s2 * (rx + ry), s2 * (ry + rz), s2 * (rz + rx)};
  float f[D_IN];
  f[0] = (float)(rx * inv_scale);
  f[1] = (float)(ry * inv_scale);
  f[2] = (float)(rz * inv_scale);
  f[3] = (float)normals[3 * i];
  f[4] = (float)normals[3 * i + 1];
  f[5] = (float)normals[3 * i + 2];
  f[6] = (float)(k * inv_kmax);
  f[7] = (float)(k * inv_kmax * k * inv_kmax);
#pragma unroll
  for (int j = 0; j < 7; ++j) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double th = k * (0.5 * (q + 1)) * proj[j];
      th = remainder(th, 2.0 * kPi);
      float sv, cv;
      sincosf((float)th, &sv, &cv);
      f[8 + 2 * (4 * j + q)] = cv;
      f[9 + 2 * (4 * j + q)] = sv;
    }
  }
  __align__(16) bf16 b[D_IN];
#pragma unroll
  for (int j = 0; j < D_IN; ++j) b[j] = __float2bfloat16_rn(f[j]);
  uint4* dst = reinterpret_cast<uint4*>(X + row * D_IN);
#pragma unroll
  for (int q = 0; q < D_IN / 8; ++q) dst[q] = reinterpret_cast<const uint4*>(b)[q];
  if (Xf)
    for (int j = 0; j < D_IN; ++j) Xf[row * D_IN + j] = __bfloat162float(b[j]);
}

// Demodulated surface unknown: t = u exp(-i k d.x) with u = P (hard node) or dP/dnu (soft node);
// accumulates sum |t|^2 for the target scale.
__global__ void k_targets(const cd* __restrict__ surf, const uint8_t* __restrict__ bc, const double* __restrict__ nodes,
                          int64_t N, const double* __restrict__ kv, int nk, double dx, double dy, double dz,
                          float* __restrict__ T, double* __restrict__ sumsq) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double s = 0.0;
  if (row < (int64_t)nk * N) {
    const int64_t kk = row / N, i = row % N;
    const cd u = surf[(kk * 2 + (bc[i] ? 1 : 0)) * N + i];
    double sn, cs;
    sincos(-kv[kk] * (dx * nodes[3 * i] + dy * nodes[3 * i + 1] + dz * nodes[3 * i + 2]), &sn, &cs);
    const cd t = cmul(u, cd{cs, sn});
    T[2 * row] = (float)t.re;
    T[2 * row + 1] = (float)t.im;
    s = t.re * t.re + t.im * t.im;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(sumsq, s);
}

__global__ void k_scale(float* __restrict__ x, int64_t n, float s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= s;
}

// Inference head: x0[row] = tscale (y0 + i y1) exp(i k d.x_i), row = kk N + i.  Warp per row.
__global__ void k_head_predict(const bf16* __restrict__ H3, int64_t M, int64_t N, const float* __restrict__ theta,
                               const double* __restrict__ nodes, const double* __restrict__ kv, double dx, double dy,
                               double dz, double tscale, cd* __restrict__ x0, float* __restrict__ Y) {
  const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= M) return;
  const int c = lane * 8;
  __align__(16) bf16 hb[8];
  *reinterpret_cast<uint4*>(hb) = *reinterpret_cast<const uint4*>(H3 + row * W_H + c);
  float y0 = 0.f, y1 = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float h = __bfloat162float(hb[j]);
    y0 = fmaf(theta[OFF_W4 + c + j], h, y0);
    y1 = fmaf(theta[OFF_W4 + W_H + c + j], h, y1);
  }
  for (int o = 16; o > 0; o >>= 1) {
    y0 += __shfl_xor_sync(0xffffffffu, y0, o);
    y1 += __shfl_xor_sync(0xffffffffu, y1, o);
  }
  if (lane != 0) return;
  y0 += theta[OFF_B4];
  y1 += theta[OFF_B4 + 1];
  if (Y) {
    Y[2 * row] = y0;
    Y[2 * row + 1] = y1;
  }
  if (x0) {
    const int64_t i = row % N;
    double sn, cs;
    sincos(kv[row / N] * (dx * nodes[3 * i] + dy * nodes[3 * i + 1] + dz * nodes[3 * i + 2]), &sn, &cs);
    x0[row] = cscale(cmul(cd{(double)y0, (double)y1}, cd{cs, sn}), tscale);
  }
}

}  // namespace mlp

// =============================================================================================
// Host side
// =============================================================================================
using namespace mlp;

struct MlpState {
  float* theta = nullptr;  // FP32 master parameters
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  bf16 *w1 = nullptr, *w2 = nullptr, *w3 = nullptr, *w2t = nullptr, *w3t = nullptr;
  int64_t* step = nullptr;  // device step counter
  float* loss = nullptr;    // device loss accumulator
  int32_t* err = nullptr;   // device error flags of the tensor-core kernels
  bool has_params = false;
  double tscale = 1.0;      // target scale of the trained network
  double kmax = 0.0;        // wavenumber normalisation of the feature map
  // activations / minibatch buffers, sized for `cap` rows
  int64_t cap = 0;
  bf16 *X0 = nullptr, *X0T = nullptr, *H1 = nullptr, *H1T = nullptr, *H2 = nullptr, *H2T = nullptr, *H3 = nullptr;
  bf16 *dZ3 = nullptr, *dZ3T = nullptr, *dZ2 = nullptr, *dZ2T = nullptr, *dZ1T = nullptr;
  float* Tb = nullptr;
  void* block = nullptr;    // one allocation for all of the above
  // training set
  bf16* Xall = nullptr;
  float* Tall = nullptr;
  int32_t* idx = nullptr;
  int64_t rows_all = 0, idx_cap = 0;
  void* dset = nullptr;
};

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

static int cuda_ok(cudaError_t e, const char* what) { return e == cudaSuccess ? BIE_OK : cuda_fail(e, what); }

// Prepares the tensor-core GEMMs' shared-memory limit (outside any stream capture).
static int prepare_gemm_attrs() {
  BIE_CUDA_TRY(cudaFuncSetAttribute(k_gemm<256, EPI_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    gemm_smem_bytes<256>()));
  BIE_CUDA_TRY(cudaFuncSetAttribute(k_gemm<256, EPI_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    gemm_smem_bytes<256>()));
  BIE_CUDA_TRY(cudaFuncSetAttribute(k_gemm<256, EPI_WGRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    gemm_smem_bytes<256>()));
  BIE_CUDA_TRY(cudaFuncSetAttribute(k_gemm<64, EPI_WGRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    gemm_smem_bytes<64>()));
  return BIE_OK;
}

static int mlp_state(bie_ctx* c, MlpState** out) {
  if (!c->mlp) {
    BIE_TRY(prepare_gemm_attrs());
    MlpState* s = new MlpState();
    c->mlp = s;  // freed by mlp_free even if an allocation below fails
    const size_t P = (size_t)NPARAM;
    BIE_TRY(dev_alloc(c, (void**)&s->theta, P * 4));
    BIE_TRY(dev_alloc(c, (void**)&s->grad, P * 4));
    BIE_TRY(dev_alloc(c, (void**)&s->m, P * 4));
    BIE_TRY(dev_alloc(c, (void**)&s->v, P * 4));
    BIE_TRY(dev_alloc(c, (void**)&s->w1, W_H * D_IN * 2));
    BIE_TRY(dev_alloc(c, (void**)&s->w2, W_H * W_H * 2));
    BIE_TRY(dev_alloc(c, (void**)&s->w3, W_H * W_H * 2));
    BIE_TRY(dev_alloc(c, (void**)&s->w2t, W_H * W_H * 2));
    BIE_TRY(dev_alloc(c, (void**)&s->w3t, W_H * W_H * 2));
    BIE_TRY(dev_alloc(c, (void**)&s->step, 64));
    BIE_TRY(dev_alloc(c, (void**)&s->loss, 64));
    BIE_TRY(dev_alloc(c, (void**)&s->err, 64));
    BIE_CUDA_TRY(cudaMemsetAsync(s->grad, 0, P * 4, c->stream));
    BIE_CUDA_TRY(cudaMemsetAsync(s->m, 0, P * 4, c->stream));
    BIE_CUDA_TRY(cudaMemsetAsync(s->v, 0, P * 4, c->stream));
    BIE_CUDA_TRY(cudaMemsetAsync(s->step, 0, 64, c->stream));
    BIE_CUDA_TRY(cudaMemsetAsync(s->err, 0, 64, c->stream));
  }
  *out = c->mlp;
  return BIE_OK;
}

void mlp_free(bie_ctx* c) {
  MlpState* s = c->mlp;
  if (!s) return;
  for (void* p : {(void*)s->theta, (void*)s->grad, (void*)s->m, (void*)s->v, (void*)s->w1, (void*)s->w2, (void*)s->w3,
                  (void*)s->w2t, (void*)s->w3t, (void*)s->step, (void*)s->loss, (void*)s->err, s->block, s->dset})
    dev_free(c, p);
  delete s;
  c->mlp = nullptr;
}

static int ensure_act(bie_ctx* c, MlpState* s, int64_t rows) {
  rows = round_up(std::max<int64_t>(rows, 128), 128);
  if (rows <= s->cap) return BIE_OK;
  if (s->block) {
    dev_free(c, s->block);
    s->block = nullptr;
    s->cap = 0;
  }
  const size_t r = (size_t)rows;
  const size_t bytes = r * (2 * D_IN * 2 + 10 * W_H * 2 + 2 * 4) + 16 * 256;
  BIE_TRY(dev_alloc(c, (void**)&s->block, bytes));
  char* q = (char*)s->block;
  auto take = [&](size_t b) { char* p = q; q += (b + 255) & ~(size_t)255; return (void*)p; };
  s->X0 = (bf16*)take(r * D_IN * 2);
  s->X0T = (bf16*)take(r * D_IN * 2);
  s->H1 = (bf16*)take(r * W_H * 2);
  s->H1T = (bf16*)take(r * W_H * 2);
  s->H2 = (bf16*)take(r * W_H * 2);
  s->H2T = (bf16*)take(r * W_H * 2);
  s->H3 = (bf16*)take(r * W_H * 2);
  s->dZ3 = (bf16*)take(r * W_H * 2);
  s->dZ3T = (bf16*)take(r * W_H * 2);
  s->dZ2 = (bf16*)take(r * W_H * 2);
  s->dZ2T = (bf16*)take(r * W_H * 2);
  s->dZ1T = (bf16*)take(r * W_H * 2);
  s->Tb = (float*)take(r * 2 * 4);
  s->cap = rows;
  return BIE_OK;
}

// ---- tensor maps ---------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

int tcx::make_map_bf16_2d(CUtensorMap* m, const void* base, uint64_t cols, uint64_t rows, uint64_t pitch_elems,
                          uint32_t box_cols, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return fail(BIE_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if (box_cols * 2 != 128 || ((uintptr_t)base & 15) || (pitch_elems * 2) % 16)
    return fail(BIE_ERR_INVALID_ARG, "BF16 tensor map: unaligned base or pitch");
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {pitch_elems * 2};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(BIE_ERR_CUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
  return BIE_OK;
}

// C[M][NT] = A[M][K] B[NT][K]^T with A (pitch lda) and B (pitch ldb) BF16 row-major.
template <int NT, int EPI>
static int gemm(bie_ctx* c, MlpState* s, const bf16* A, int64_t M, int64_t K, int64_t lda, const bf16* B, int64_t ldb,
                const Epi& ep, int kslices = 1) {
  if (K % KC != 0 || M <= 0) return fail(BIE_ERR_INVALID_ARG, "learned warm start: GEMM shape");
  CUtensorMap ma, mb;
  BIE_TRY(tcx::make_map_bf16_2d(&ma, A, (uint64_t)K, (uint64_t)M, (uint64_t)lda, KC, BM));
  BIE_TRY(tcx::make_map_bf16_2d(&mb, B, (uint64_t)K, (uint64_t)NT, (uint64_t)ldb, KC, NT));
  const int kc_total = (int)(K / KC);
  kslices = std::max(1, std::min(kslices, kc_total));
  const int kpc = (kc_total + kslices - 1) / kslices;
  kslices = (kc_total + kpc - 1) / kpc;  // every slice holds at least one chunk
  dim3 g((unsigned)((M + BM - 1) / BM), (unsigned)kslices);
  BIE_LAUNCH(k_gemm<NT, EPI><<<g, 128, gemm_smem_bytes<NT>(), c->stream>>>(ma, mb, (int)M, kpc, kc_total, ep, s->err));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

static int wgrad_slices(int64_t Bp) {
  const int kc = (int)(Bp / KC);
  return std::max(1, std::min(kc / 2, 64));
}

// Forward through the three hidden layers for rows X0[0..M) (X0 already staged, M <= cap);
// the transposed copies are written only when `train`.
static int forward_hidden(bie_ctx* c, MlpState* s, int64_t M, int64_t ldT, bool train) {
  Epi e1{s->theta + OFF_B1, nullptr, s->H1, train ? s->H1T : nullptr, ldT, nullptr};
  BIE_TRY((gemm<256, EPI_FWD>(c, s, s->X0, M, D_IN, D_IN, s->w1, D_IN, e1)));
  Epi e2{s->theta + OFF_B2, nullptr, s->H2, train ? s->H2T : nullptr, ldT, nullptr};
  BIE_TRY((gemm<256, EPI_FWD>(c, s, s->H1, M, W_H, W_H, s->w2, W_H, e2)));
  Epi e3{s->theta + OFF_B3, nullptr, s->H3, nullptr, ldT, nullptr};
  BIE_TRY((gemm<256, EPI_FWD>(c, s, s->H2, M, W_H, W_H, s->w3, W_H, e3)));
  return BIE_OK;
}

// One loss/gradient evaluation on the staged minibatch (X0, X0T, Tb with B valid rows of Bp);
// the gradient is accumulated into s->grad (which must be zero on entry).
static int loss_grad_staged(bie_ctx* c, MlpState* s, int64_t B, int64_t Bp) {
  BIE_TRY(forward_hidden(c, s, Bp, Bp, true));
  BIE_LAUNCH(k_head_train<<<(unsigned)(Bp / 32), 256, 0, c->stream>>>(s->H3, (int)B, (int)Bp, s->theta, s->Tb,
                                                                      1.0f / (float)B, s->grad, s->dZ3, s->dZ3T, Bp,
                                                                      s->loss));
  const int ks = wgrad_slices(Bp);
  Epi w3{nullptr, nullptr, nullptr, nullptr, 0, s->grad + OFF_W3};
  BIE_TRY((gemm<256, EPI_WGRAD>(c, s, s->dZ3T, W_H, Bp, Bp, s->H2T, Bp, w3, ks)));
  Epi b2{nullptr, s->H2, s->dZ2, s->dZ2T, Bp, nullptr};
  BIE_TRY((gemm<256, EPI_BWD>(c, s, s->dZ3, Bp, W_H, W_H, s->w3t, W_H, b2)));
  Epi w2{nullptr, nullptr, nullptr, nullptr, 0, s->grad + OFF_W2};
  BIE_TRY((gemm<256, EPI_WGRAD>(c, s, s->dZ2T, W_H, Bp, Bp, s->H1T, Bp, w2, ks)));
  Epi b1{nullptr, s->H1, nullptr, s->dZ1T, Bp, nullptr};
  BIE_TRY((gemm<256, EPI_BWD>(c, s, s->dZ2, Bp, W_H, W_H, s->w2t, W_H, b1)));
  Epi w1{nullptr, nullptr, nullptr, nullptr, 0, s->grad + OFF_W1};
  BIE_TRY((gemm<64, EPI_WGRAD>(c, s, s->dZ1T, W_H, Bp, Bp, s->X0T, Bp, w1, ks)));
  BIE_LAUNCH(k_bias_grad<<<(2 * W_H) / 8, 256, 0, c->stream>>>(s->dZ1T, s->dZ2T, Bp, (int)B, s->grad));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

static int check_err(bie_ctx* c, MlpState* s) {
  int32_t e = 0;
  BIE_CUDA_TRY(cudaMemcpyAsync(&e, s->err, 4, cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (e) {
    BIE_CUDA_TRY(cudaMemsetAsync(s->err, 0, 4, c->stream));
    return fail(BIE_ERR_TIMEOUT, "learned warm start: a tensor-core wait gave up (flags " + std::to_string(e) + ")");
  }
  return BIE_OK;
}

static void geometry_frame(bie_ctx* c, double centre[3], double& scale) {
  const int64_t N = c->N;
  centre[0] = centre[1] = centre[2] = 0.0;
  for (int64_t i = 0; i < N; ++i)
    for (int a = 0; a < 3; ++a) centre[a] += c->h_nodes[3 * i + a] / (double)N;
  scale = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double r2 = 0.0;
    for (int a = 0; a < 3; ++a) r2 += (c->h_nodes[3 * i + a] - centre[a]) * (c->h_nodes[3 * i + a] - centre[a]);
    scale = std::max(scale, std::sqrt(r2));
  }
  if (!(scale > 0.0)) scale = 1.0;
}

// Features of all (k, node) rows into X (BF16, [nk*N][64]); optional FP32 copy.
static int features(bie_ctx* c, const double* kdev, int nk, bf16* X, float* Xf) {
  MlpState* s;
  BIE_TRY(mlp_state(c, &s));
  const double kmax = c->mlp_kmax > 0.0 ? c->mlp_kmax : s->kmax;
  if (!(kmax > 0.0)) return fail(BIE_ERR_STATE, "learned warm start: no wavenumber scale (train first or set learned.kmax)");
  double ctr[3], scale;
  geometry_frame(c, ctr, scale);
  const int64_t rows = (int64_t)nk * c->N;
  BIE_LAUNCH(k_features<<<(unsigned)((rows + 127) / 128), 128, 0, c->stream>>>(
      c->nodes, c->normals, c->N, kdev, nk, c->dir[0], c->dir[1], c->dir[2], ctr[0], ctr[1], ctr[2], 1.0 / scale,
      1.0 / kmax, X, Xf));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

static int upload_k(bie_ctx* c, const double* k, int64_t nk, double** kdev) {
  BIE_TRY(ensure_buf(c, c->work3, (size_t)nk * sizeof(double) + 256));
  *kdev = (double*)c->work3.p;
  BIE_CUDA_TRY(cudaMemcpyAsync(*kdev, k, nk * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  return BIE_OK;
}

// ---- public pieces (called from capi.cu) ---------------------------------------------------------
int mlp_set_params(bie_ctx* c, const float* theta_host) {
  MlpState* s;
  BIE_TRY(mlp_state(c, &s));
  BIE_CUDA_TRY(cudaMemcpyAsync(s->theta, theta_host, NPARAM * 4, cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaMemsetAsync(s->m, 0, NPARAM * 4, c->stream));
  BIE_CUDA_TRY(cudaMemsetAsync(s->v, 0, NPARAM * 4, c->stream));
  BIE_CUDA_TRY(cudaMemsetAsync(s->grad, 0, NPARAM * 4, c->stream));
  BIE_CUDA_TRY(cudaMemsetAsync(s->step, 0, 8, c->stream));
  BIE_LAUNCH(k_sync_weights<<<256, 256, 0, c->stream>>>(s->theta, s->w1, s->w2, s->w3, s->w2t, s->w3t));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  s->has_params = true;
  return BIE_OK;
}

int mlp_get_params(bie_ctx* c, float* theta_host) {
  MlpState* s;
  BIE_TRY(mlp_state(c, &s));
  if (!s->has_params) return fail(BIE_ERR_STATE, "learned warm start: no parameters yet");
  BIE_CUDA_TRY(cudaMemcpyAsync(theta_host, s->theta, NPARAM * 4, cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

// Glorot-uniform weights, zero biases, from a splitmix64 stream seeded by `seed`.
int mlp_init_params(bie_ctx* c, uint64_t seed) {
  std::vector<float> th((size_t)NPARAM, 0.0f);
  uint64_t st = seed;
  auto next = [&]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  auto fill = [&](int64_t off, int fo, int fi) {
    const double a = std::sqrt(6.0 / (fo + fi));
    for (int64_t i = 0; i < (int64_t)fo * fi; ++i) th[off + i] = (float)((2.0 * next() - 1.0) * a);
  };
  fill(OFF_W1, W_H, D_IN);
  fill(OFF_W2, W_H, W_H);
  fill(OFF_W3, W_H, W_H);
  fill(OFF_W4, D_OUT, W_H);
  return mlp_set_params(c, th.data());
}

int mlp_features_api(bie_ctx* c, const double* k, int64_t nk, float* phi) {
  if (!c->has_geom) return fail(BIE_ERR_STATE, "no geometry");
  if (nk <= 0) return BIE_OK;
  MlpState* s;
  BIE_TRY(mlp_state(c, &s));
  double* kdev;
  BIE_TRY(upload_k(c, k, nk, &kdev));
  const int64_t rows = nk * c->N;
  BIE_TRY(ensure_act(c, s, rows));
  // the BF16 rows land in the activation block (H1 region is large enough: rows*256 >= rows*64)
  BIE_TRY(features(c, kdev, (int)nk, s->H1, phi));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

static int stage_f32(bie_ctx* c, MlpState* s, const float* X, const float* T, int64_t B, int64_t Bp) {
  // X (FP32 [B][64]) -> BF16 rows in H1 (scratch), then gather into X0/X0T/Tb with zero padding
  BIE_LAUNCH(k_f32_to_bf16<<<256, 256, 0, c->stream>>>(X, B * D_IN, s->H1));
  if (T) {
    BIE_CUDA_TRY(cudaMemcpyAsync(s->dZ2, T, B * 2 * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
  } else {
    BIE_CUDA_TRY(cudaMemsetAsync(s->dZ2, 0, B * 2 * sizeof(float), c->stream));
  }
  BIE_LAUNCH(k_gather<<<(unsigned)(Bp / 32), 256, 0, c->stream>>>(s->H1, reinterpret_cast<const float*>(s->dZ2), nullptr,
                                                                  (int)B, (int)Bp, s->X0, s->X0T, s->Tb, nullptr));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int mlp_forward_api(bie_ctx* c, const float* X, int64_t B, float* Y) {
  MlpState* s;
  BIE_TRY(mlp_state(c, &s));
  if (!s->has_params) return fail(BIE_ERR_STATE, "learned warm start: no parameters yet");
  if (B <= 0) return BIE_OK;
  const int64_t Bp = round_up(B, 128);
  BIE_TRY(ensure_act(c, s, Bp));
  BIE_TRY(stage_f32(c, s, X, nullptr, B, Bp));
  BIE_TRY(forward_hidden(c, s, B, Bp, false));
  BIE_LAUNCH(k_head_predict<<<(unsigned)((B + 7) / 8), 256, 0, c->stream>>>(s->H3, B, 1, s->theta, nullptr, nullptr, 0,
                                                                           0, 0, 1.0, nullptr, Y));
  BIE_CUDA_TRY(cudaGetLastError());
  return check_err(c, s);
}

int mlp_loss_grad_api(bie_ctx* c, const float* X, const float* T, int64_t B, float* grad, float* loss) {
  MlpState* s;
  BIE_TRY(mlp_state(c, &s));
  if (!s->has_params) return fail(BIE_ERR_STATE, "learned warm start: no parameters yet");
  if (B <= 0) return fail(BIE_ERR_INVALID_ARG, "empty batch");
  const int64_t Bp = round_up(B, 128);
  BIE_TRY(ensure_act(c, s, Bp));
  BIE_CUDA_TRY(cudaMemsetAsync(s->grad, 0, NPARAM * 4, c->stream));
  BIE_CUDA_TRY(cudaMemsetAsync(s->loss, 0, 4, c->stream));
  BIE_TRY(stage_f32(c, s, X, T, B, Bp));
  BIE_TRY(loss_grad_staged(c, s, B, Bp));
  if (grad) BIE_CUDA_TRY(cudaMemcpyAsync(grad, s->grad, NPARAM * 4, cudaMemcpyDeviceToDevice, c->stream));
  if (loss) BIE_CUDA_TRY(cudaMemcpyAsync(loss, s->loss, 4, cudaMemcpyDeviceToDevice, c->stream));
  return check_err(c, s);
}

int mlp_adam_api(bie_ctx* c, const float* grad, double lr) {
  MlpState* s;
  BIE_TRY(mlp_state(c, &s));
  if (!s->has_params) return fail(BIE_ERR_STATE, "learned warm start: no parameters yet");
  BIE_CUDA_TRY(cudaMemcpyAsync(s->grad, grad, NPARAM * 4, cudaMemcpyDeviceToDevice, c->stream));
  int64_t t = 0;
  BIE_CUDA_TRY(cudaMemcpyAsync(&t, s->step, 8, cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  t += 1;
  BIE_CUDA_TRY(cudaMemcpyAsync(s->step, &t, 8, cudaMemcpyHostToDevice, c->stream));
  BIE_LAUNCH(k_adam<<<256, 256, 0, c->stream>>>(s->theta, s->grad, s->m, s->v, s->step, (float)lr, (float)lr, 0, 0.9f,
                                                0.999f, 1e-8f, s->w1, s->w2, s->w3, s->w2t, s->w3t));
  BIE_CUDA_TRY(cudaGetLastError());
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

// Training on the solutions of `nk` wavenumbers: surf (device, c128 [nk][2][N]).  Every epoch
// visits the rows in a fresh seeded order in minibatches of c->mlp_batch; one epoch's launches
// are captured once in a CUDA graph and replayed.  loss_hist (host, optional) receives the mean
// minibatch loss of every epoch.
int mlp_train(bie_ctx* c, const double* k, int64_t nk, const cd* surf, int epochs, float* loss_hist) {
  if (!c->has_geom) return fail(BIE_ERR_STATE, "no geometry");
  if (nk <= 0 || epochs < 0) return fail(BIE_ERR_INVALID_ARG, "learned warm start: nothing to train on");
  MlpState* s;
  BIE_TRY(mlp_state(c, &s));
  if (!s->has_params) BIE_TRY(mlp_init_params(c, (uint64_t)c->mlp_seed));
  const int64_t N = c->N, rows = nk * N;
  double kmax = 0.0;
  for (int64_t i = 0; i < nk; ++i) kmax = std::max(kmax, k[i]);
  s->kmax = c->mlp_kmax > 0.0 ? c->mlp_kmax : kmax;
  const int64_t Bv = std::min<int64_t>(round_up(std::max<int64_t>(c->mlp_batch, 128), 128), round_up(rows, 128));
  const int64_t nmb = std::max<int64_t>(1, rows / Bv);  // full minibatches per epoch (rows beyond are skipped)
  const int64_t Bp = Bv;
  const int64_t Bvalid = std::min<int64_t>(Bv, rows);
  // training set: features + scaled targets
  if (s->dset) {
    dev_free(c, s->dset);
    s->dset = nullptr;
  }
  const size_t xb = ((size_t)rows * D_IN * 2 + 255) & ~(size_t)255, tb = ((size_t)rows * 8 + 255) & ~(size_t)255;
  const size_t ib = ((size_t)nmb * Bp * 4 + 255) & ~(size_t)255;
  BIE_TRY(dev_alloc(c, (void**)&s->dset, xb + tb + ib + 256 + (size_t)nk * 8 + 256));
  s->Xall = (bf16*)s->dset;
  s->Tall = (float*)((char*)s->dset + xb);
  s->idx = (int32_t*)((char*)s->dset + xb + tb);
  double* sumsq = (double*)((char*)s->dset + xb + tb + ib);
  double* kdev = (double*)((char*)s->dset + xb + tb + ib + 256);
  BIE_CUDA_TRY(cudaMemcpyAsync(kdev, k, nk * 8, cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaMemsetAsync(sumsq, 0, 8, c->stream));
  BIE_TRY(features(c, kdev, (int)nk, s->Xall, nullptr));
  BIE_LAUNCH(k_targets<<<(unsigned)((rows + 255) / 256), 256, 0, c->stream>>>(
      surf, c->bc, c->nodes, N, kdev, (int)nk, c->dir[0], c->dir[1], c->dir[2], s->Tall, sumsq));
  double ss = 0.0;
  BIE_CUDA_TRY(cudaMemcpyAsync(&ss, sumsq, 8, cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  s->tscale = ss > 0.0 ? std::sqrt(ss / (double)rows) : 1.0;
  BIE_LAUNCH(k_scale<<<256, 256, 0, c->stream>>>(s->Tall, rows * 2, (float)(1.0 / s->tscale)));
  BIE_TRY(ensure_act(c, s, Bp));
  // one epoch of launches
  const int64_t total_steps = (int64_t)epochs * nmb;
  auto epoch_body = [&]() -> int {
    for (int64_t b = 0; b < nmb; ++b) {
      BIE_LAUNCH(k_gather<<<(unsigned)(Bp / 32), 256, 0, c->stream>>>(s->Xall, s->Tall, s->idx + b * Bp, (int)Bvalid,
                                                                      (int)Bp, s->X0, s->X0T, s->Tb, s->step));
      BIE_TRY(loss_grad_staged(c, s, Bvalid, Bp));
      BIE_LAUNCH(k_adam<<<(unsigned)((NPARAM + 255) / 256), 256, 0, c->stream>>>(
          s->theta, s->grad, s->m, s->v, s->step, (float)c->mlp_lr, (float)c->mlp_lr_min, total_steps, 0.9f, 0.999f,
          1e-8f, s->w1, s->w2, s->w3, s->w2t, s->w3t));
    }
    BIE_CUDA_TRY(cudaGetLastError());
    return BIE_OK;
  };
  BIE_CUDA_TRY(cudaMemsetAsync(s->grad, 0, NPARAM * 4, c->stream));
  std::vector<int32_t> perm((size_t)rows), idx((size_t)nmb * Bp);
  uint64_t st = (uint64_t)c->mlp_seed * 0x2545F4914F6CDD1Dull + 17;
  auto rnd = [&]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  cudaGraphExec_t exec = nullptr;
  int graph_nodes = 0;
  int rc = BIE_OK;
  for (int e = 0; e < epochs && rc == BIE_OK; ++e) {
    for (int64_t i = 0; i < rows; ++i) perm[i] = (int32_t)i;
    for (int64_t i = rows - 1; i > 0; --i) std::swap(perm[i], perm[(int64_t)(rnd() % (uint64_t)(i + 1))]);
    for (int64_t b = 0; b < nmb; ++b)
      for (int64_t r = 0; r < Bp; ++r) idx[b * Bp + r] = r < Bvalid ? perm[(b * Bvalid + r) % rows] : 0;
    rc = cuda_ok(cudaMemcpyAsync(s->idx, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice, c->stream), "idx upload");
    if (rc != BIE_OK) break;
    rc = cuda_ok(cudaMemsetAsync(s->loss, 0, 4, c->stream), "loss reset");
    if (rc != BIE_OK) break;
    if (c->mlp_graph) {
      if (!exec) {
        cudaGraph_t graph = nullptr;
        const int64_t before = bie_kernel_launches();
        cudaStream_t saved = nullptr;
        rc = capture_begin(c, &saved);
        if (rc != BIE_OK) break;
        const int body = epoch_body();
        const int re = capture_end(c, saved, &graph);
        if (body != BIE_OK || re != BIE_OK) {
          rc = body != BIE_OK ? body : re;
          if (graph) cudaGraphDestroy(graph);
          break;
        }
        graph_nodes = (int)(bie_kernel_launches() - before);
        rc = cuda_ok(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate");
        cudaGraphDestroy(graph);
        if (rc != BIE_OK) break;
        uncount_launches(graph_nodes);  // captured, not launched: counted per replay below
      }
      rc = cuda_ok(cudaGraphLaunch(exec, c->stream), "graph launch");
      count_launches(graph_nodes);
    } else {
      rc = epoch_body();
    }
    if (rc == BIE_OK && loss_hist) {
      float L = 0.f;
      rc = cuda_ok(cudaMemcpyAsync(&L, s->loss, 4, cudaMemcpyDeviceToHost, c->stream), "loss read");
      if (rc == BIE_OK) rc = cuda_ok(cudaStreamSynchronize(c->stream), "sync");
      loss_hist[e] = L / (float)nmb;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  BIE_TRY(rc);
  return check_err(c, s);
}

// Initial guesses x0 (device c128 [nk][N]) for wavenumbers kdev[nk] from the trained network.
int mlp_predict_dev(bie_ctx* c, const double* kdev, int nk, cd* x0) {
  MlpState* s;
  BIE_TRY(mlp_state(c, &s));
  if (!s->has_params) return fail(BIE_ERR_STATE, "learned warm start: not trained");
  const int64_t N = c->N;
  // rows processed in chunks that fit the activation buffers
  const int64_t chunk = std::max<int64_t>(128, std::min<int64_t>((int64_t)nk * N, (int64_t)1 << 18));
  const int64_t per = std::max<int64_t>(1, chunk / N);  // wavenumbers per chunk
  BIE_TRY(ensure_act(c, s, per * N));
  for (int64_t k0 = 0; k0 < nk; k0 += per) {
    const int nkc = (int)std::min<int64_t>(per, nk - k0);
    const int64_t rows = (int64_t)nkc * N;
    BIE_TRY(features(c, kdev + k0, nkc, s->X0, nullptr));
    BIE_TRY(forward_hidden(c, s, rows, rows, false));
    BIE_LAUNCH(k_head_predict<<<(unsigned)((rows + 7) / 8), 256, 0, c->stream>>>(
        s->H3, rows, N, s->theta, c->nodes, kdev + k0, c->dir[0], c->dir[1], c->dir[2], s->tscale, x0 + k0 * N,
        nullptr));
  }
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int mlp_predict_api(bie_ctx* c, const double* k, int64_t nk, cd* x0) {
  if (!c->has_geom) return fail(BIE_ERR_STATE, "no geometry");
  if (nk <= 0) return BIE_OK;
  double* kdev;
  BIE_TRY(upload_k(c, k, nk, &kdev));
  BIE_TRY(mlp_predict_dev(c, kdev, (int)nk, x0));
  MlpState* s;
  BIE_TRY(mlp_state(c, &s));
  return check_err(c, s);
}

}  // namespace bie
