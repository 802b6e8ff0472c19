// lu_tc.cu -- blocked complex LU ("solved using a direct method", Sec. 4) with the trailing update
// A22 -= L21 U12 on the 5th-generation tensor cores (tcgen05, TF32 operands, FP32 accumulation in
// tensor memory).  Panel factorisation with partial pivoting and the U12 solve run on the CUDA
// cores (lu.cu); the update, a genuine dense contraction, runs here.
//
// Complex product by four real products (4M):  Re = Lr Ur - Li Ui,  Im = Lr Ui + Li Ur, with three
// FP32 accumulators in TMEM (T1 = Lr Ur, T2 = Li Ui, T3 = Lr Ui + Li Ur), combined in the epilogue.
//
// CTA = 128 threads, output tile 128 rows x 64 complex columns, K = panel width (64).  All threads
// stage L21 / U12 from global memory into shared memory in the canonical K-major, no-swizzle
// UMMA layout (8-row x 16-byte core matrices, K-adjacent core matrices 128 B apart, 8-row groups
// 1024 B apart), de-interleaving real/imaginary parts, transposing U12 and rounding to TF32.
// Thread 0 issues the MMAs (M = 128, N = 64, K = 8 each) and commits them to an mbarrier; the four
// warps then read their 32 TMEM lanes each (tcgen05.ld 32x32b) and update A22 in place.
// Shared memory 96 KB and TMEM 256 columns per CTA: two CTAs per SM, so one CTA's staging and
// epilogue overlap the other's MMAs.
#include "bie_common.cuh"

namespace bie {

int lu_panel_steps32(bie_ctx* c, cf* A, int batch, int n, int ld, int64_t bstride, int p0, int w, int32_t* piv,
                     int32_t* info);

namespace tc {

constexpr int BM = 128;           // rows per tile (TMEM lanes)
constexpr int BN = 64;            // complex columns per tile
constexpr int NB = 64;            // panel width = K of the update
constexpr int KC = 32;            // K per staged chunk (128 bytes of TF32 per row)
constexpr int NCH = NB / KC;      // chunks
constexpr int A_CHUNK = BM * KC * 4;   // 16 KB
constexpr int B_CHUNK = BN * KC * 4;   // 8 KB
constexpr int SMEM_LR = 0;
constexpr int SMEM_LI = SMEM_LR + NCH * A_CHUNK;
constexpr int SMEM_UR = SMEM_LI + NCH * A_CHUNK;
constexpr int SMEM_UI = SMEM_UR + NCH * B_CHUNK;
constexpr int SMEM_BYTES = SMEM_UI + NCH * B_CHUNK;  // 96 KB
constexpr int TMEM_COLS = 256;    // T1 [0,64), T2 [64,128), T3 [128,192)
constexpr uint32_t SPIN_LIMIT = 1u << 26;

// byte offset of element (row r, k) inside one K-chunk of a canonical K-major operand tile
__device__ __forceinline__ uint32_t canon_off(int r, int k) {
  return (uint32_t)(((r >> 3) * 8 + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// UMMA shared-memory descriptor: start, LBO (K-direction core stride), SBO (8-row group stride),
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major, N = 64, M = 128.
__host__ __device__ constexpr uint32_t make_idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(addr), "r"(phase)
      : "memory");
  return ok != 0;
}

// grid: (ceil(rem / BN), ceil(rem / BM), batch).  Updates A[r][c] for r, c in [p0 + NB, n).
__global__ void __launch_bounds__(128, 2) k_update_tc(float* __restrict__ A, int64_t bstride, int n, int ld, int p0,
                                                     int32_t* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kbase = p0, rbase = p0 + NB;
  const int R0 = rbase + blockIdx.y * BM, C0 = rbase + blockIdx.x * BN;
  float* M = A + (int64_t)blockIdx.z * bstride * 2;  // interleaved complex: 2 floats per entry

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }

  // ---- stage L21 (BM x NB) and U12^T (BN x NB) as TF32, real and imaginary planes ----
  // L rows are contiguous in k: each float4 holds entries k, k+1 of one row.
  for (int t = tid; t < BM * (NB / 2); t += 128) {
    const int r = t / (NB / 2), k = (t % (NB / 2)) * 2;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    const int gr = R0 + r;
    if (gr < n) v = *reinterpret_cast<const float4*>(M + 2 * ((int64_t)gr * ld + kbase + k));
    const int ch = k / KC, kk = k % KC;
    const uint32_t off = canon_off(r, kk);
    *reinterpret_cast<float2*>(sm + SMEM_LR + ch * A_CHUNK + off) = make_float2(to_tf32(v.x), to_tf32(v.z));
    *reinterpret_cast<float2*>(sm + SMEM_LI + ch * A_CHUNK + off) = make_float2(to_tf32(v.y), to_tf32(v.w));
  }
  // U12 rows (index k) are contiguous in the column index c: each float4 holds columns c, c+1.
  for (int t = tid; t < NB * (BN / 2); t += 128) {
    const int k = t / (BN / 2), cc = (t % (BN / 2)) * 2;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    const int gc = C0 + cc;
    const float* src = M + 2 * ((int64_t)(kbase + k) * ld + gc);
    if (gc + 1 < n) v = *reinterpret_cast<const float4*>(src);
    else if (gc < n) v = make_float4(src[0], src[1], 0.f, 0.f);
    const int ch = k / KC, kk = k % KC;
    const uint32_t o0 = canon_off(cc, kk), o1 = canon_off(cc + 1, kk);
    *reinterpret_cast<float*>(sm + SMEM_UR + ch * B_CHUNK + o0) = to_tf32(v.x);
    *reinterpret_cast<float*>(sm + SMEM_UI + ch * B_CHUNK + o0) = to_tf32(v.y);
    *reinterpret_cast<float*>(sm + SMEM_UR + ch * B_CHUNK + o1) = to_tf32(v.z);
    *reinterpret_cast<float*>(sm + SMEM_UI + ch * B_CHUNK + o1) = to_tf32(v.w);
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (tid == 0) {
    const uint32_t idesc = make_idesc();
    const uint32_t base = smem_u32(sm);
    for (int ch = 0; ch < NCH; ++ch)
      for (int s = 0; s < KC / 8; ++s) {
        const uint32_t ka = ch * A_CHUNK + s * 256, kb = ch * B_CHUNK + s * 256;
        const uint64_t ar = make_desc(base + SMEM_LR + ka, 128, 1024);
        const uint64_t ai = make_desc(base + SMEM_LI + ka, 128, 1024);
        const uint64_t br = make_desc(base + SMEM_UR + kb, 128, 1024);
        const uint64_t bi = make_desc(base + SMEM_UI + kb, 128, 1024);
        const uint32_t acc = (ch | s) ? 1u : 0u;
        mma_tf32(tmem + 0, ar, br, idesc, acc);    // T1 = Lr Ur
        mma_tf32(tmem + 64, ai, bi, idesc, acc);   // T2 = Li Ui
        mma_tf32(tmem + 128, ar, bi, idesc, acc);  // T3 = Lr Ui
        mma_tf32(tmem + 128, ai, br, idesc, 1u);   //    + Li Ur
      }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(&mbar))
                 : "memory");
  }
  // wait for the MMAs (bounded: a lost arrival sets the error flag instead of hanging)
  bool ok = false;
  for (uint32_t it = 0; it < SPIN_LIMIT; ++it)
    if (mbar_try_wait(smem_u32(&mbar), 0)) { ok = true; break; }
  if (!ok && lane == 0) atomicOr(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  if (ok) {
    const int r = warp * 32 + lane;
    const int gr = R0 + r;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int cc = 0; cc < BN; cc += 16) {
      float t1[16], t2[16], t3[16];
      tmem_ld16(trow + cc, t1);
      tmem_ld16(trow + 64 + cc, t2);
      tmem_ld16(trow + 128 + cc, t3);
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (gr < n) {
        float* dst = M + 2 * ((int64_t)gr * ld + C0 + cc);
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          if (C0 + cc + j + 1 < n) {
            float4 v = *reinterpret_cast<float4*>(dst + 2 * j);
            v.x -= t1[j] - t2[j];
            v.y -= t3[j];
            v.z -= t1[j + 1] - t2[j + 1];
            v.w -= t3[j + 1];
            *reinterpret_cast<float4*>(dst + 2 * j) = v;
          } else if (C0 + cc + j < n) {
            dst[2 * j] -= t1[j] - t2[j];
            dst[2 * j + 1] -= t3[j];
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
}

}  // namespace tc

size_t lu_tc_scratch_bytes(int batch, int n) { return 256; }

int lu_factor_tc(bie_ctx* c, cf* A, int batch, int n, int ld, int64_t bstride, int32_t* piv, int32_t* info,
                 void* scratch, size_t scratch_bytes) {
  using namespace tc;
  if (ld % 2 != 0 || bstride % 2 != 0) return fail(BIE_ERR_INVALID_ARG, "tcgen05 LU needs even ld and batch stride");
  int32_t* err = (int32_t*)scratch;
  BIE_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), c->stream));
  BIE_CUDA_TRY(cudaFuncSetAttribute(k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
  for (int p0 = 0; p0 < n; p0 += NB) {
    const int w = std::min(NB, n - p0);
    BIE_TRY(lu_panel_steps32(c, A, batch, n, ld, bstride, p0, w, piv, info));
    const int rem = n - p0 - w;
    if (rem > 0) {
      dim3 g((unsigned)((rem + BN - 1) / BN), (unsigned)((rem + BM - 1) / BM), (unsigned)batch);
      BIE_LAUNCH(k_update_tc<<<g, 128, SMEM_BYTES, c->stream>>>(reinterpret_cast<float*>(A), bstride, n, ld, p0, err));
    }
  }
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int lu_tc_error(bie_ctx* c, void* scratch, int32_t* out) {
  BIE_CUDA_TRY(cudaMemcpy(out, scratch, sizeof(int32_t), cudaMemcpyDeviceToHost));
  return BIE_OK;
}

}  // namespace bie
