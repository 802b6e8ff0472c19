// lu_tc.cu -- blocked complex LU (the direct solver of Sec. 4) with the trailing update
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
#include <cuda.h>
#include <cudaTypedefs.h>

#include "bie_common.cuh"

namespace bie {

int lu_panel_steps32(bie_ctx* c, cf* A, int batch, int n, int ld, int64_t bstride, int p0, int w, int32_t* piv,
                     int32_t* info, int tend, void* coop, int32_t* err, float* ub, int64_t ub_stride, int krow,
                     int koff, bool* emitted);
size_t lu_coop_scratch_bytes(int batch);
int lu_trsm_rows32(bie_ctx* c, cf* A, int batch, int n, int ld, int64_t bstride, int p0, int w, int jlo, float* ub,
                   int64_t ub_stride, int krow, int koff, bool* emitted);

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

// ==============================================================================================
// Version 2: persistent, warp-specialised, TMA-fed update with the complex product written as a
// real GEMM on the interleaved storage (real embedding):
//   C_int (m x 2n reals) -= L_int (m x 2K reals) * B,  B = [[ur, ui], [-ui, ur]] per complex u,
// so L21 is consumed exactly as stored (re, im, re, im, ...) and B^T (2n x 2K, K-major) is built
// once per panel by k_build_ub.  Roles: warp 0 lane 0 issues TMA loads of 128-row x 32-float boxes
// (128-byte swizzle) into a 4-stage ring; warp 1 lane 0 issues tcgen05.mma (M = 128, N = 128,
// K = 8, TF32) and commits each stage back to the producer and each finished tile to the
// epilogue; warps 2-5 move the tile out of TMEM (double-buffered accumulators, 2 x 128 columns)
// and subtract it from A22, overlapping the next tile's MMAs.  Every wait is bounded and sets an
// error flag instead of hanging.
// ==============================================================================================
namespace tc2 {

constexpr int BM = 128;                  // rows per tile
constexpr int KCH = 32;                  // floats per 128-byte swizzle row
constexpr int STAGES = 4;
constexpr int A_STAGE = BM * KCH * 4;    // 16 KB
// BNR: real columns per tile, 256 (128 complex; the default) or 128, a template parameter of
// the kernel ("mixed.lu_tile"): B stage BNR x 32 floats (one 128-row TMA box per 128 rows),
// two BNR-column accumulators in TMEM
template <int BNR>
constexpr int b_stage() { return BNR * KCH * 4; }
template <int BNR>
constexpr int smem_bytes() { return STAGES * (A_STAGE + b_stage<BNR>()) + 2 * A_STAGE + 1024; }  // ring + 2 boxes
constexpr int NTHREADS = 192;
constexpr uint32_t SPIN = 1u << 22;

struct alignas(8) Bars {
  uint64_t full[STAGES], empty[STAGES], acc_full[2], acc_empty[2];
  uint32_t tmem_slot;
  uint32_t abort;  // set by an epilogue warp whose wait gave up
};

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}
// bounded wait; returns false (and raises the error flag) when the limit is reached
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int32_t* err) {
  for (uint32_t i = 0; i < SPIN; ++i)
    if (tc::mbar_try_wait(a, parity)) return true;
  atomicOr(err, 2);
  return false;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::
          "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
// K-major operand in the 128-byte-swizzled canonical layout: 8-row atoms of 128 B, atoms 1024 B
// apart (SBO), leading offset unused, descriptor version 1, layout type 2 (SWIZZLE_128B).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
template <int BNR>
__host__ __device__ constexpr uint32_t idesc_m128() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BNR >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// B^T of the real embedding for nrows (<= 64) rows of U (rows u0 .. u0+nrows-1 of A, row
// k = u0 + kk): for column c in [cb, cend), B^T rows 2 (c - cb) and 2 (c - cb) + 1 get, at floats
// koff + 2 kk, [ur, -ui] and [ui, ur] (rows `krow` floats long).  Columns at or past n are zero.
// grid (ceil((cend - cb) / 32), batch)
__global__ void __launch_bounds__(256) k_build_ub(const float* __restrict__ A, int64_t bstride, int n, int ld, int u0,
                                                  int cb, int cend, float* __restrict__ ub, int64_t ub_stride,
                                                  int krow, int koff, int nrows) {
  __shared__ float2 t[tc::NB][33];
  const int z = blockIdx.y;
  const int c0 = blockIdx.x * 32;
  const float* M = A + (int64_t)z * bstride * 2;
  for (int e = threadIdx.x; e < nrows * 32; e += blockDim.x) {  // U rows k, columns cb + c0 .. +31
    const int k = e / 32, cc = e % 32;
    const int gc = cb + c0 + cc;
    float2 u = make_float2(0.f, 0.f);
    if (gc < n && gc < cend) u = *reinterpret_cast<const float2*>(M + 2 * ((int64_t)(u0 + k) * ld + gc));
    t[k][cc] = u;
  }
  __syncthreads();
  float* out = ub + (int64_t)z * ub_stride;
  for (int e = threadIdx.x; e < 32 * nrows; e += blockDim.x) {
    const int cc = e / nrows, k = e % nrows;
    if (cb + c0 + cc >= cend) continue;
    const float2 u = t[k][cc];
    const int64_t r = 2 * (int64_t)(c0 + cc);
    const float ur = tc::to_tf32(u.x), ui = tc::to_tf32(u.y);  // round to nearest TF32 once here
    *reinterpret_cast<float2*>(out + r * krow + koff + 2 * k) = make_float2(ur, -ui);
    *reinterpret_cast<float2*>(out + (r + 1) * krow + koff + 2 * k) = make_float2(ui, ur);
  }
}

// One update region: rows [r0, r1), complex columns [c0, c1) of every matrix get
//   A -= L U,  L = A[rows][kc0 .. kc0 + 16 nchk),  U from the B^T map (row 2 (c - ub_c0)),
// in tiles of 128 rows x 64 complex columns.  Rows at or past r1 inside the last row tile are
// left unchanged (their share of the tile is zeroed before the reduction).
struct Region {
  int r0, r1, c0, c1, kc0, nchk, ub_c0, ntm, ntn;
};

// Tile order: per matrix, bands of kBand column tiles, row tiles in order within a band, columns
// innermost.  The CTAs in flight then share a few bands' U operand and a few row tiles' L operand
// (at N = 8004, K = 512 the row-major order kept every column tile's U in flight, 62 MB per
// matrix, which the A22 traffic evicted from L2: 1.5 GB of operand re-reads from DRAM per launch).
constexpr int kBand = 8;
__device__ __forceinline__ void tile_coords(int tile, int ntm, int ntn, int& z, int& tm, int& tn) {
  const int per = ntm * ntn;
  z = tile / per;
  const int r = tile - z * per;
  const int full = ntn / kBand;  // bands of kBand columns; the last band may be narrower
  const int g = r / (ntm * kBand);
  if (g < full) {
    const int w = r - g * ntm * kBand;
    tm = w / kBand;
    tn = g * kBand + (w - tm * kBand);
  } else {
    const int gw = ntn - full * kBand;
    const int w = r - full * ntm * kBand;
    tm = w / gw;
    tn = full * kBand + (w - tm * gw);
  }
}

template <int BNR>
__global__ void __launch_bounds__(NTHREADS, 1) k_update_tc2(const __grid_constant__ CUtensorMap tmA,
                                                           const __grid_constant__ CUtensorMap tmB, int batch,
                                                           const Region rg, int32_t* __restrict__ err) {
  static_assert(BNR == 128 || BNR == 256, "tile of 128 or 256 real columns");
  constexpr int B_STAGE = b_stage<BNR>();
  constexpr int TMEM_COLS = 2 * BNR;  // two BNR-column accumulators (a power of two >= 32)
  extern __shared__ unsigned char smraw[];
  __shared__ Bars bar;
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  const uint32_t smA = tc::smem_u32(sm), smB = smA + STAGES * A_STAGE;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto baddr = [&](const uint64_t& b) { return tc::smem_u32(&b); };
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(baddr(bar.full[s]), 1);
      mbar_init(baddr(bar.empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(baddr(bar.acc_full[a]), 1);
      mbar_init(baddr(bar.acc_empty[a]), 4);
    }
    bar.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tc::smem_u32(&bar.tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = bar.tmem_slot;
  const int ntm = rg.ntm, ntn = rg.ntn, nchk = rg.nchk;
  const int ntiles = batch * ntm * ntn;

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer ----
      uint32_t it = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        int z, tm, tn;
        tile_coords(tile, ntm, ntn, z, tm, tn);
        for (int ch = 0; ch < nchk && ok; ++ch, ++it) {
          const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
          ok = mbar_wait(baddr(bar.empty[s]), ph ^ 1, err);
          if (!ok) break;
          mbar_expect_tx(baddr(bar.full[s]), A_STAGE + B_STAGE);
          tma_load_3d(smA + s * A_STAGE, &tmA, 2 * rg.kc0 + ch * KCH, rg.r0 + tm * BM, z, baddr(bar.full[s]));
          const int yb = 2 * (rg.c0 - rg.ub_c0) + tn * BNR;  // B^T rows of the tile, boxes of BM rows
#pragma unroll
          for (int bx = 0; bx < BNR / BM; ++bx)
            tma_load_3d(smB + s * B_STAGE + bx * BM * KCH * 4, &tmB, ch * KCH, yb + bx * BM, z, baddr(bar.full[s]));
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer ----
      const uint32_t idesc = idesc_m128<BNR>();
      uint32_t it = 0, ti = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++ti) {
        const uint32_t a = ti & 1, aph = (ti >> 1) & 1;
        ok = mbar_wait(baddr(bar.acc_empty[a]), aph ^ 1, err);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t d = tmem + a * BNR;
        for (int ch = 0; ch < nchk && ok; ++ch, ++it) {
          const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
          ok = mbar_wait(baddr(bar.full[s]), ph, err);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
          for (int k = 0; k < KCH / 8; ++k)
            tc::mma_tf32(d, desc_sw128(smA + s * A_STAGE + k * 32), desc_sw128(smB + s * B_STAGE + k * 32), idesc,
                         (ch | k) ? 1u : 0u);
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                           baddr(bar.empty[s]))
                       : "memory");
        }
        if (ok)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                           baddr(bar.acc_full[a]))
                       : "memory");
      }
    }
  } else {  // ---- epilogue warps 2..5: TMEM lane quarter = warp % 4 ----
    // Each 32-column chunk of the accumulator is negated into a 128-byte-swizzled staging box
    // (two boxes, alternating) and added to A22 by a TMA reduction: the L2 performs the
    // read-modify-write, the epilogue never waits on global loads.
    const int q = warp & 3;
    const int rt = q * 32 + lane;
    const bool leader = (warp == 2 && lane == 0);
    const uint32_t smD = smB + STAGES * B_STAGE;  // 2 x 16 KB, 1024-aligned
    uint32_t ti = 0, nb = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++ti) {
      int z, tm, tn;
      tile_coords(tile, ntm, ntn, z, tm, tn);
      const uint32_t a = ti & 1, aph = (ti >> 1) & 1;
      // every epilogue warp reaches the named barrier once per tile, then all leave together if
      // any of them gave up waiting (no warp may be left alone at a later barrier)
      if (!mbar_wait(baddr(bar.acc_full[a]), aph, err)) bar.abort = 1;
      asm volatile("bar.sync 1, 128;\n" ::: "memory");
      if (*(volatile uint32_t*)&bar.abort) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const int gr0 = rg.r0 + tm * BM;
      const int gc0 = 2 * (rg.c0 + tn * (BNR / 2));  // first real column of the tile
      const int gc_end = 2 * rg.c1;                   // chunks at or past it are not reduced
      const bool keep = gr0 + rt < rg.r1;             // rows past r1 add zero
      const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + a * BNR;
#pragma unroll 1
      for (int cc = 0; cc < BNR; cc += 32, ++nb) {
        // chunks at or past the region's last column are neither staged nor reduced (the same
        // decision in all four warps; nb counts only the chunks that commit a reduction, so the
        // box written next was read by the reduction two commits back)
        if (gc0 + cc >= gc_end) break;
        float v[32];
        tmem_ld32(ta + cc, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        const uint32_t box = smD + (nb & 1) * A_STAGE;
        // the reduction issued two chunks ago read this box: wait until it has
        if (leader) asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
        asm volatile("bar.sync 1, 128;\n" ::: "memory");
#pragma unroll
        for (int c4 = 0; c4 < 8; ++c4) {
          const uint32_t off = (uint32_t)rt * 128 + (uint32_t)((c4 ^ (rt & 7)) * 16);
          const float4 o = keep ? make_float4(-v[4 * c4], -v[4 * c4 + 1], -v[4 * c4 + 2], -v[4 * c4 + 3])
                                : make_float4(0.f, 0.f, 0.f, 0.f);
          asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(box + off), "f"(o.x), "f"(o.y), "f"(o.z),
                       "f"(o.w)
                       : "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("bar.sync 1, 128;\n" ::: "memory");
        if (leader) {
          asm volatile(
              "cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(
                  reinterpret_cast<uint64_t>(&tmA)),
              "r"(gc0 + cc), "r"(gr0), "r"(z), "r"(box)
              : "memory");
          asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(baddr(bar.acc_empty[a]));
    }
    if (leader) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link-time libcuda).
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

static int make_map_3d(CUtensorMap* m, const void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1_bytes,
                       uint64_t s2_bytes) {
  auto fn = encode_fn();
  if (!fn) return fail(BIE_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {s1_bytes, s2_bytes};
  const cuuint32_t box[3] = {(cuuint32_t)KCH, (cuuint32_t)BM, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(BIE_ERR_CUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
  return BIE_OK;
}

}  // namespace tc2

// Version 3 (the default): the update of version 2, with the trailing update deferred over an
// outer block of NBO columns (c->lu_block: 128, 256 or 512, i.e. 2, 4 or 8 64-column panels), so
// that A22 is read and written once per NBO columns instead of once per 64 (at NBO = 256 the
// intensity is 8 x 256 / 16 = 128 flop per byte of A22):
//   for each outer block [P0, E):
//     for each panel [p0, p0 + 64): factor it; swap rows in every column; U = L11^{-1} A for the
//       block's columns right of the panel; update rows below the panel in the block's columns
//       right of it (K = 64).  Columns at or past E get only the swaps.
//     U12 (block rows, columns >= E) by block forward substitution: for each 64-row block b,
//       A_b -= L_b,<b U_<b (K = 64 b), then U_b = L_bb^{-1} A_b.
//     A22 (rows and columns >= E) -= L21 U12 with K = 256.
constexpr int kMaxLuBlock = 512;

// Columns of the deferred update: the "mixed.lu_block" option, or (0, the default) 512 from
// N = 8192 on -- at 256 the A22 traffic (16 B per complex entry per block) would bound the update
// of such matrices below the TF32 rate (128 flop per byte at 256, 256 at 512) -- and 256 below.
int lu_block_for(const bie_ctx* c, int n) {
  if (c->lu_block > 0) return c->lu_block;
  return n >= 8192 ? 512 : 256;
}

size_t lu_tc_scratch_bytes(int batch, int n, int block) {
  // error flag, the cooperative panel's scratch, B^T for one 64-row panel (128 floats per row)
  // and for one outer block (2 NBO)
  if (block < tc::NB || block > kMaxLuBlock) block = kMaxLuBlock;
  return 256 + ((lu_coop_scratch_bytes(batch) + 255) & ~(size_t)255) +
         (size_t)batch * 2 * n * (2 * tc::NB + 2 * block) * sizeof(float);
}

int lu_factor_tc(bie_ctx* c, cf* A, int batch, int n, int ld, int64_t bstride, int32_t* piv, int32_t* info,
                 void* scratch, size_t scratch_bytes) {
  using namespace tc;
  if (ld % 64 != 0 || bstride % 2 != 0) return fail(BIE_ERR_INVALID_ARG, "tcgen05 LU needs ld % 64 == 0 and even batch stride");
  int32_t* err = (int32_t*)scratch;
  BIE_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), c->stream));
  void* coop = (char*)scratch + 256;
  const int ver = c->tc_version;
  const int NBO = lu_block_for(c, n);
  // panel width of the deferred version (32 or 64; versions 1 and 2 use 64)
  const int nb = (ver >= 3 && c->lu_panel == 32) ? 32 : NB;
  if (NBO % NB != 0 || NBO < NB || NBO > kMaxLuBlock) return fail(BIE_ERR_INVALID_ARG, "LU block must be 128, 256 or 512");
  float* ub = reinterpret_cast<float*>((char*)coop + ((lu_coop_scratch_bytes(batch) + 255) & ~(size_t)255));
  const int kr = 2 * nb;                                // reals along K of one panel's B^T
  const int64_t ub_stride = (int64_t)2 * n * kr;        // floats per matrix, one panel
  float* ubo = ub + (int64_t)batch * ub_stride;
  const int64_t ubo_stride = (int64_t)2 * n * (2 * NBO);  // floats per matrix, outer block
  const float* Af = reinterpret_cast<const float*>(A);
  CUtensorMap mA, mB, mBo;
  int nsm = 148;
  if (ver >= 2) {
    if (scratch_bytes < lu_tc_scratch_bytes(batch, n, ver >= 3 ? NBO : NB))
      return fail(BIE_ERR_STATE, "tcgen05 scratch too small");
    BIE_TRY(tc2::make_map_3d(&mA, A, (uint64_t)2 * n, (uint64_t)n, (uint64_t)batch, (uint64_t)2 * ld * 4,
                             (uint64_t)bstride * 8));
    BIE_TRY(tc2::make_map_3d(&mB, ub, (uint64_t)kr, (uint64_t)2 * n, (uint64_t)batch, (uint64_t)kr * 4,
                             (uint64_t)ub_stride * 4));
    BIE_TRY(tc2::make_map_3d(&mBo, ubo, (uint64_t)2 * NBO, (uint64_t)2 * n, (uint64_t)batch, (uint64_t)2 * NBO * 4,
                             (uint64_t)ubo_stride * 4));
    BIE_TRY((set_smem_max(tc2::k_update_tc2<256>)));
    BIE_TRY((set_smem_max(tc2::k_update_tc2<128>)));
    BIE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
  } else {
    BIE_TRY((set_smem_max(k_update_tc)));
  }
  // B^T of U rows u0 .. u0+rows-1, columns [cb, cend), into the panel or the outer-block buffer
  auto build = [&](int u0, int cb, int cend, bool outer, int koff, int rows) -> int {
    if (cend <= cb) return BIE_OK;
    dim3 gb((unsigned)((cend - cb + 31) / 32), (unsigned)batch);
    BIE_LAUNCH(tc2::k_build_ub<<<gb, 256, 0, c->stream>>>(Af, bstride, n, ld, u0, cb, cend, outer ? ubo : ub,
                                                          outer ? ubo_stride : ub_stride, outer ? 2 * NBO : kr,
                                                          koff, rows));
    return BIE_OK;
  };
  // tile width in real columns ("mixed.lu_tile": 256 = 128 complex columns, or 128)
  const int bnr = c->lu_tile == 128 ? 128 : 256;
  auto update = [&](int r0, int r1, int c0, int c1, int kc0, int kcols, bool outer, int ub_c0) -> int {
    if (r1 <= r0 || c1 <= c0 || kcols <= 0) return BIE_OK;
    tc2::Region rg{r0, r1, c0, c1, kc0, 2 * kcols / tc2::KCH, ub_c0, (r1 - r0 + tc2::BM - 1) / tc2::BM,
                   (c1 - c0 + bnr / 2 - 1) / (bnr / 2)};
    const int ntiles = rg.ntm * rg.ntn * batch;
    const int grid = std::min(ntiles, nsm);
    if (bnr == 256)
      BIE_LAUNCH(tc2::k_update_tc2<256><<<grid, tc2::NTHREADS, tc2::smem_bytes<256>(), c->stream>>>(
          mA, outer ? mBo : mB, batch, rg, err));
    else
      BIE_LAUNCH(tc2::k_update_tc2<128><<<grid, tc2::NTHREADS, tc2::smem_bytes<128>(), c->stream>>>(
          mA, outer ? mBo : mB, batch, rg, err));
    return BIE_OK;
  };
  if (ver >= 3) {
    for (int P0 = 0; P0 < n; P0 += NBO) {
      const int E = std::min(n, P0 + NBO);
      for (int p0 = P0; p0 < E; p0 += nb) {
        const int w = std::min(nb, E - p0), q = p0 + w;
        // the U solve of the block's columns right of the panel also writes their B^T (64-row
        // panels); otherwise the build pass does
        bool emitted = false;
        BIE_TRY(lu_panel_steps32(c, A, batch, n, ld, bstride, p0, w, piv, info, E, coop, err, ub, ub_stride, kr, 0,
                                 &emitted));
        if (q < E) {  // then w == nb (E - P0 is a multiple of nb unless E == n)
          if (!emitted) BIE_TRY(build(p0, q, E, false, 0, w));
          BIE_TRY(update(q, n, q, E, p0, w, false, q));
        }
      }
      if (E >= n) continue;  // E - P0 == NBO from here on
      for (int b = 0; b < NBO / nb; ++b) {
        const int Rb = P0 + b * nb;
        BIE_TRY(update(Rb, Rb + nb, E, n, P0, b * nb, true, E));
        bool emitted = false;
        BIE_TRY(lu_trsm_rows32(c, A, batch, n, ld, bstride, Rb, nb, E, ubo, ubo_stride, 2 * NBO, 2 * nb * b, &emitted));
        if (!emitted) BIE_TRY(build(Rb, E, n, true, 2 * nb * b, nb));
      }
      BIE_TRY(update(E, n, E, n, P0, NBO, true, E));
    }
    BIE_CUDA_TRY(cudaGetLastError());
    return BIE_OK;
  }
  for (int p0 = 0; p0 < n; p0 += NB) {
    const int w = std::min(NB, n - p0);
    BIE_TRY(lu_panel_steps32(c, A, batch, n, ld, bstride, p0, w, piv, info, n, coop, err, nullptr, 0, 0, 0, nullptr));
    const int rem = n - p0 - w;
    if (rem <= 0) continue;
    if (ver == 2) {
      BIE_TRY(build(p0, p0 + NB, n, false, 0, NB));
      BIE_TRY(update(p0 + NB, n, p0 + NB, n, p0, NB, false, p0 + NB));
    } else {
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
