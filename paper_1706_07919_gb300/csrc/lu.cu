// lu.cu -- batched dense complex LU with partial pivoting and triangular solves (the direct solver
// of Sec. 4), right-looking and blocked:
//   for each panel of width nb:  factor the panel (pivot = largest modulus, lowest row on ties),
//   apply its row swaps to the other columns, U12 = L11^{-1} A12, A22 -= L21 U12.
// Matrices are row-major with leading dimension ld, batched with stride `bstride` elements.
// This file holds the panel, swap/TRSM and SIMT-GEMM kernels in FP64 and FP32; the tensor-core
// (tcgen05, TF32) trailing update lives in lu_tc.cu.
#include "bie_common.cuh"

namespace bie {

template <class S> struct Cx { S re, im; };
template <class S> __device__ __forceinline__ Cx<S> cx_mul(Cx<S> a, Cx<S> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class S> __device__ __forceinline__ Cx<S> cx_div(Cx<S> a, Cx<S> b) {
  S d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// ---- panel factorisation: one CTA per matrix, columns p0 .. p0+nb-1, rows p0 .. n-1 ----------
template <class S>
__global__ void __launch_bounds__(512) k_panel(Cx<S>* __restrict__ A, int64_t bstride, int n, int ld, int p0,
                                               int nb, int32_t* __restrict__ piv, int32_t* __restrict__ info) {
  Cx<S>* M = A + (int64_t)blockIdx.x * bstride;
  int32_t* pv = piv + (int64_t)blockIdx.x * n;
  __shared__ S red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_piv;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int pend = min(p0 + nb, n);
  for (int c = p0; c < pend; ++c) {
    // pivot: largest |a_rc|^2 over r >= c, lowest row on ties
    S best = -1;
    int bi = n;
    for (int r = c + tid; r < n; r += nt) {
      Cx<S> v = M[(int64_t)r * ld + c];
      S m = v.re * v.re + v.im * v.im;
      if (m > best) { best = m; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      S ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      best = lane < nw ? red_v[lane] : (S)-1;
      bi = lane < nw ? red_i[lane] : n;
      for (int o = 16; o > 0; o >>= 1) {
        S ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        s_piv = bi;
        pv[c] = bi;
        if (!(best > 0) && info) atomicOr(info + blockIdx.x, 1);
      }
    }
    __syncthreads();
    const int p = s_piv;
    if (p != c && p < n)  // swap rows c and p inside the panel columns
      for (int j = p0 + tid; j < pend; j += nt) {
        Cx<S> t = M[(int64_t)c * ld + j];
        M[(int64_t)c * ld + j] = M[(int64_t)p * ld + j];
        M[(int64_t)p * ld + j] = t;
      }
    __syncthreads();
    const Cx<S> d = M[(int64_t)c * ld + c];
    const bool ok = (d.re != 0 || d.im != 0);
    // scale the column and update the rest of the panel (rank-1), one row per thread
    for (int r = c + 1 + tid; r < n; r += nt) {
      Cx<S> l = M[(int64_t)r * ld + c];
      if (ok) l = cx_div(l, d);
      M[(int64_t)r * ld + c] = l;
      for (int j = c + 1; j < pend; ++j) {
        Cx<S> u = M[(int64_t)c * ld + j];
        Cx<S> a = M[(int64_t)r * ld + j];
        a.re -= l.re * u.re - l.im * u.im;
        a.im -= l.re * u.im + l.im * u.re;
        M[(int64_t)r * ld + j] = a;
      }
    }
    __syncthreads();
  }
}

// ---- leaf-recursive panel: a leaf of `lw` columns factored in shared memory ------------------
// One CTA (1024 threads) per matrix holds rows c0..n-1 of columns c0..c0+lw-1, factors them with
// partial pivoting (largest modulus, lowest row on ties), writes them back, applies the leaf's
// row swaps to the other columns of the panel [p0, p0+w) and solves the leaf's U block for the
// panel columns right of the leaf, then updates the panel columns right of the leaf in the rows
// below it.  The leaf is stored column by column in shared memory (element (r, c) at
// c * rows + r), so that threads walking the rows touch consecutive words.
template <class S>
__global__ void __launch_bounds__(1024) k_leaf(Cx<S>* __restrict__ A, int64_t bstride, int n, int ld, int p0, int w,
                                               int c0, int lw, int32_t* __restrict__ piv, int32_t* __restrict__ info,
                                               int fuse) {
  extern __shared__ unsigned char smem_raw[];
  Cx<S>* L = reinterpret_cast<Cx<S>*>(smem_raw);  // [lw][rows]
  __shared__ S red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_piv[16];
  Cx<S>* M = A + (int64_t)blockIdx.x * bstride;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int rows = n - c0;
  // global-memory loops are unrolled so that several loads per thread are in flight
  // 16-byte accesses need an even element index: even ld, batch stride, c0 and leaf width (the
  // last also keeps the U block below, at element rows * lw of the shared array, 16-byte aligned)
  const bool pairs = sizeof(S) == 4 && ((ld | bstride | c0 | lw) & 1) == 0;
  if (pairs) {  // FP32: 16-byte loads of column pairs
    const int hl = lw >> 1;
#pragma unroll 4
    for (int t = tid; t < rows * hl; t += nt) {
      const int r = t / hl, c = 2 * (t - r * hl);
      const float4 v = *reinterpret_cast<const float4*>(&M[(int64_t)(c0 + r) * ld + c0 + c]);
      L[c * rows + r] = Cx<S>{(S)v.x, (S)v.y};
      L[(c + 1) * rows + r] = Cx<S>{(S)v.z, (S)v.w};
    }
  } else {
#pragma unroll 4
    for (int t = tid; t < rows * lw; t += nt) {
      const int r = t / lw, c = t - r * lw;
      L[c * rows + r] = M[(int64_t)(c0 + r) * ld + c0 + c];
    }
  }
  __syncthreads();
  for (int c = 0; c < lw; ++c) {
    S best = -1;
    int bi = rows;
    for (int r = c + tid; r < rows; r += nt) {
      const Cx<S> v = L[c * rows + r];
      const S m = v.re * v.re + v.im * v.im;
      if (m > best) { best = m; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const S ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      best = lane < nw ? red_v[lane] : (S)-1;
      bi = lane < nw ? red_i[lane] : rows;
      for (int o = 16; o > 0; o >>= 1) {
        const S ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        if (bi >= rows) bi = c;
        s_piv[c] = bi;
        piv[(int64_t)blockIdx.x * n + c0 + c] = c0 + bi;
        if (!(best > 0) && info) atomicOr(info + blockIdx.x, 1);
      }
    }
    __syncthreads();
    const int p = s_piv[c];
    if (p != c && tid < lw) {
      const Cx<S> t = L[tid * rows + c];
      L[tid * rows + c] = L[tid * rows + p];
      L[tid * rows + p] = t;
    }
    __syncthreads();
    const Cx<S> d = L[c * rows + c];
    const bool ok = (d.re != 0 || d.im != 0);
    for (int r = c + 1 + tid; r < rows; r += nt) {
      Cx<S> l = L[c * rows + r];
      if (ok) l = cx_div(l, d);
      L[c * rows + r] = l;
      for (int j = c + 1; j < lw; ++j) {
        const Cx<S> u = L[j * rows + c];
        Cx<S> a = L[j * rows + r];
        a.re -= l.re * u.re - l.im * u.im;
        a.im -= l.re * u.im + l.im * u.re;
        L[j * rows + r] = a;
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < rows * lw; t += nt) {
    const int r = t / lw, c = t - r * lw;
    M[(int64_t)(c0 + r) * ld + c0 + c] = L[c * rows + r];
  }
  // other panel columns: their rows c0 .. c0+lw-1 are staged in shared memory (X, [lw][wall]),
  // where each column's thread applies the leaf's swaps in order (rows below the leaf are swapped
  // in global memory) and solves the U block right of the leaf; then X is written back.  The
  // dependent chains of a column run on shared memory, not on global-memory round trips.
  const int pend = min(p0 + w, n);
  const int wall = pend - p0;
  Cx<S>* X = L + (size_t)rows * lw;  // [lw][wall]
  for (int t = tid; t < lw * wall; t += nt) {
    const int s = t / wall, jj = t - s * wall, j = p0 + jj;
    if (j >= c0 && j < c0 + lw) continue;
    X[t] = M[(int64_t)(c0 + s) * ld + j];
  }
  __syncthreads();
  for (int jj = tid; jj < wall; jj += nt) {
    const int j = p0 + jj;
    if (j >= c0 && j < c0 + lw) continue;
    for (int s = 0; s < lw; ++s) {
      const int p = s_piv[s];  // leaf-relative row, p >= s
      if (p != s) {
        const Cx<S> t = X[s * wall + jj];
        if (p < lw) {
          X[s * wall + jj] = X[p * wall + jj];
          X[p * wall + jj] = t;
        } else {
          Cx<S>& g = M[(int64_t)(c0 + p) * ld + j];
          X[s * wall + jj] = g;
          g = t;
        }
      }
    }
    if (j >= c0 + lw)
      for (int s = 1; s < lw; ++s) {
        Cx<S> v = X[s * wall + jj];
        for (int t = 0; t < s; ++t) {
          const Cx<S> l = L[t * rows + s];
          const Cx<S> xt = X[t * wall + jj];
          v.re -= l.re * xt.re - l.im * xt.im;
          v.im -= l.re * xt.im + l.im * xt.re;
        }
        X[s * wall + jj] = v;
      }
    for (int s = 0; s < lw; ++s) M[(int64_t)(c0 + s) * ld + j] = X[s * wall + jj];
  }
  // rows below the leaf, panel columns right of it: A -= L_leaf U_leaf, with the leaf's L and its
  // just-solved U block (in X) from shared memory; consecutive threads take consecutive columns
  // of a row (coalesced read-modify-write)
  const int cs = c0 + lw, wr = pend - cs;
  if (fuse && wr > 0 && rows > lw) {
    __syncthreads();  // every column's U block is complete in X
    const Cx<S>* U = X + (cs - p0);  // U[s * wall + j]: row c0 + s, column cs + j
    if (pairs && (wr & 1) == 0 && (wall & 1) == 0) {  // cs = c0 + lw and cs - p0 are even too
      // FP32: a thread takes two adjacent columns (one 16-byte load and store), several in flight
      const int hw = wr >> 1;
#pragma unroll 4
      for (int t = tid; t < (rows - lw) * hw; t += nt) {
        const int rr = t / hw, j = 2 * (t - rr * hw), r = lw + rr;
        float4* mp = reinterpret_cast<float4*>(&M[(int64_t)(c0 + r) * ld + cs + j]);
        float4 a = *mp;
        for (int s2 = 0; s2 < lw; ++s2) {
          const Cx<S> l = L[s2 * rows + r];
          const float4 u = *reinterpret_cast<const float4*>(&U[s2 * wall + j]);
          a.x -= l.re * u.x - l.im * u.y;
          a.y -= l.re * u.y + l.im * u.x;
          a.z -= l.re * u.z - l.im * u.w;
          a.w -= l.re * u.w + l.im * u.z;
        }
        *mp = a;
      }
    } else {
#pragma unroll 4
      for (int t = tid; t < (rows - lw) * wr; t += nt) {
        const int rr = t / wr, j = t - rr * wr, r = lw + rr;
        Cx<S>& m = M[(int64_t)(c0 + r) * ld + cs + j];
        Cx<S> a = m;
        for (int s2 = 0; s2 < lw; ++s2) {
          const Cx<S> l = L[s2 * rows + r], u = U[s2 * wall + j];
          a.re -= l.re * u.re - l.im * u.im;
          a.im -= l.re * u.im + l.im * u.re;
        }
        m = a;
      }
    }
  }
}

// Rows below the leaf, panel columns right of it: A -= L_leaf U_leaf (K = lw <= 16), as its own
// launch for small batches (the leaf kernel has one CTA per matrix).  One warp per row, lanes over the (<= 64) columns so that the read-modify-write of A coalesces;
// the row's lw entries of L are broadcast.  grid (ceil(rows / 64), batch), block 256 (8 warps, 8
// rows each).
template <class S>
__global__ void __launch_bounds__(256) k_leaf_update(Cx<S>* __restrict__ A, int64_t bstride, int n, int ld, int p0,
                                                     int w, int c0, int lw) {
  __shared__ Cx<S> U[16 * 64];
  Cx<S>* M = A + (int64_t)blockIdx.y * bstride;
  const int cs = c0 + lw, ce = min(p0 + w, n), wr = ce - cs;
  if (wr <= 0) return;
  for (int t = threadIdx.x; t < lw * wr; t += blockDim.x) {
    const int s = t / wr, j = t - s * wr;
    U[s * 64 + j] = M[(int64_t)(c0 + s) * ld + cs + j];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rbeg = c0 + lw + blockIdx.x * 64;
  for (int r = rbeg + warp; r < min(rbeg + 64, n); r += 8) {
    const Cx<S>* lrow = M + (int64_t)r * ld + c0;
    Cx<S> l[16];
#pragma unroll
    for (int s = 0; s < 16; ++s)
      if (s < lw) l[s] = lrow[s];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      if (j < wr) {
        S ar = 0, ai = 0;
#pragma unroll
        for (int s = 0; s < 16; ++s)
          if (s < lw) {
            const Cx<S> u = U[s * 64 + j];
            ar += l[s].re * u.re - l[s].im * u.im;
            ai += l[s].re * u.im + l[s].im * u.re;
          }
        Cx<S>& m = M[(int64_t)r * ld + cs + j];
        m.re -= ar;
        m.im -= ai;
      }
    }
  }
}

// ---- cooperative panel: several CTAs per matrix for a few tall matrices ----------------------
// With few matrices in a batch (at most half as many as co-resident CTAs) and panels taller than
// a 16-column leaf that fits one CTA's shared memory, one CTA per matrix leaves most SMs idle and
// has to narrow its leaves to a column or two.  Here `cpm` CTAs share each matrix: CTA j of
// matrix z holds rows [p0 + j ch, p0 + (j + 1) ch) of a leaf of up to 16 columns in shared memory
// (column by column), and the CTAs of one matrix agree on every pivot through records in global
// memory, one exchange per column:
//   each CTA posts its best candidate row (largest modulus, lowest row on ties) with the
//   candidate's leaf entries (CTA 0 adds row c's), the record's tag written last with release
//   semantics; one warp of every CTA polls the matrix's tags (acquire) until all carry this
//   column's, which makes the exchange its own barrier; every CTA picks the same winner p, the
//   holders of rows c and p exchange them in shared memory, and every CTA scales column c of its
//   rows and applies the rank-1 update to the rest of its leaf, finding its next candidate on the
//   way.  The records of consecutive columns alternate between two buffers, which is safe because
//   no CTA can post column c + 2 before every CTA has posted column c + 1, after reading column c.
// After a leaf, CTA 0 (its chunk holds the panel's diagonal rows: ch is a multiple of 64) applies
// the leaf's row interchanges, as one gather of the at most 2 lw rows they touch, to the panel's
// other columns and solves the leaf's U block L11^{-1} A12 for the panel columns right of the
// leaf; after a barrier (a counter in global memory) every CTA updates its rows of those
// columns, A -= L U (K = lw).
// Launched cooperatively, so that all CTAs are resident together.  Every wait is bounded: a CTA
// whose wait gives up raises the error word (bit 8) and an abort flag on which every other wait
// ends, and all CTAs leave.  Data written by other CTAs is read with L2-coherent loads.
namespace coop {
constexpr int NT = 512;
constexpr int LWMAX = 16;
constexpr int WMAX = 64;                 // panel width
constexpr uint32_t SPIN = 1u << 21;      // polls of one wait (about a second) before giving up
struct alignas(16) Cand {                // one CTA's pivot candidate for one column
  // |a|^2 of the candidate (bits of the float, -1: no row) << 32 | its row << 8 | tag: the column's
  // place in the panel + 1 (1 .. 64; 0: not written in this launch), stored last with release
  // semantics, so that one acquire load gives the whole verdict
  unsigned long long head;
  int pad[2];
  Cx<float> v[LWMAX];                    // the candidate's leaf entries
  Cx<float> d[LWMAX];                    // CTA 0: row c's leaf entries
};
// scratch: [nmat] barrier counters, abort flag, [2][grid] candidate records (zeroed before each
// launch with the counters)
inline size_t scratch_bytes(int nmat, int grid) {
  return 256 + (size_t)(nmat + 1) * 4 + 256 + 2 * (size_t)grid * sizeof(Cand) + 256;
}
}  // namespace coop
constexpr int kCoopMaxGrid = 4096;  // CTAs of one cooperative panel launch (at most)

__device__ __forceinline__ unsigned long long ld_acquire_gpu64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];\n" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ Cx<float> ldcg_cx(const Cx<float>* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}

__global__ void __launch_bounds__(coop::NT, 1) k_panel_coop(
    Cx<float>* __restrict__ A, int64_t bstride, int n, int ld, int p0, int w, int lw, int cpm, int ch,
    int32_t* __restrict__ piv, int32_t* __restrict__ info, unsigned* __restrict__ bar, unsigned* abort_flag,
    coop::Cand* __restrict__ cand, int32_t* __restrict__ err) {
  using coop::LWMAX;
  using coop::NT;
  extern __shared__ float4 coop_smem[];
  Cx<float>* S = reinterpret_cast<Cx<float>*>(coop_smem);  // [lw][ch]: leaf entry (r, t) at t * ch + r - r_lo
  Cx<float>* Ub = S + (size_t)lw * ch;                     // [LWMAX][WMAX]: the leaf's U block
  __shared__ Cx<float> s_u[LWMAX], s_d[LWMAX];             // pivot row, former row c (leaf entries)
  __shared__ float red_v[NT / 32];
  __shared__ int red_i[NT / 32];
  __shared__ int s_p, s_abort, s_m;
  __shared__ int s_piv[LWMAX], s_rows[2 * LWMAX], s_src[2 * LWMAX];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int z = blockIdx.x / cpm, j = blockIdx.x - z * cpm;
  Cx<float>* M = A + (int64_t)z * bstride;
  const int r_lo = p0 + j * ch, r_hi = min(n, r_lo + ch);  // empty when r_lo >= n
  const int pend = min(p0 + w, n);
  unsigned gen = 0;
  if (tid == 0) s_abort = 0;
  __syncthreads();
  // barrier of the cpm CTAs of matrix z; false when a wait gave up here or elsewhere.  The
  // arrival is a release (it orders the CTA's writes, gathered by bar.sync, before it), the
  // poll an acquire.
  auto barrier = [&]() -> bool {
    __syncthreads();
    if (tid == 0) {
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;\n" ::"l"(bar + z) : "memory");
      const unsigned target = (gen + 1) * (unsigned)cpm;
      bool ok = false;
      for (uint32_t it = 0; it < coop::SPIN; ++it) {
        if (ld_acquire_gpu(bar + z) >= target) { ok = true; break; }
        if (ld_acquire_gpu(abort_flag)) break;
        if (it > 16) __nanosleep(32);
      }
      if (!ok) {
        atomicOr(err, 8);
        atomicExch(abort_flag, 1u);
        s_abort = 1;
      }
      asm volatile("fence.acq_rel.gpu;\n" ::: "memory");
    }
    ++gen;
    __syncthreads();
    return s_abort == 0;
  };
  for (int c0 = p0; c0 < pend; c0 += lw) {
    const int l = min(lw, pend - c0);
    const int a = max(r_lo, c0);       // first leaf row held here
    const int nr = max(0, r_hi - a);
    for (int e = tid; e < nr * l; e += NT) {
      const int rr = e / l, t = e - rr * l;
      S[t * ch + a - r_lo + rr] = ldcg_cx(M + (int64_t)(a + rr) * ld + c0 + t);
    }
    __syncthreads();
    // this thread's candidate for the leaf's first column (later columns: found during the
    // rank-1 update of the column before)
    float best = -1.f;
    int bi = n;
    for (int r = a + tid; r < r_hi; r += NT) {
      const Cx<float> v = S[r - r_lo];
      const float m = v.re * v.re + v.im * v.im;
      if (m > best) { best = m; bi = r; }
    }
    for (int cc = 0; cc < l; ++cc) {
      const int c = c0 + cc, buf = c & 1;
      const unsigned tag = (unsigned)(c - p0) + 1u;
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
      __syncthreads();
      if (warp == 0) {
        best = lane < NT / 32 ? red_v[lane] : -1.f;
        bi = lane < NT / 32 ? red_i[lane] : n;
        for (int o = 16; o > 0; o >>= 1) {
          const float ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        coop::Cand* cd = cand + (int64_t)buf * gridDim.x + blockIdx.x;
        if (lane == 0) {  // the whole record from one thread, its head last (release)
          for (int t = 0; t < l; ++t) cd->v[t] = bi < r_hi ? S[t * ch + bi - r_lo] : Cx<float>{0.f, 0.f};
          if (c >= r_lo && c < r_hi)
            for (int t = 0; t < l; ++t) cd->d[t] = S[t * ch + c - r_lo];
          const unsigned long long head = ((unsigned long long)__float_as_uint(best) << 32) |
                                          ((unsigned long long)(unsigned)bi << 8) | tag;
          asm volatile("st.release.gpu.global.u64 [%0], %1;\n" ::"l"(&cd->head), "l"(head) : "memory");
        }
        // wait for every record of this column (bounded; the abort flag, read every 32 polls,
        // ends it too); the heads carry the candidates
        const coop::Cand* cb = cand + (int64_t)buf * gridDim.x + (int64_t)z * cpm;
        bool ok = false;
        float b2 = -1.f;
        int i2 = n, w2 = 0;
        for (uint32_t it = 0; it < coop::SPIN; ++it) {
          bool mine = true;
          float bl = -1.f;
          int il = n, wl = 0;
          for (int q = lane; q < cpm; q += 32) {
            const unsigned long long h = ld_acquire_gpu64(&cb[q].head);
            if ((unsigned)(h & 0xffu) != tag) { mine = false; break; }
            const float bq = __uint_as_float((unsigned)(h >> 32));
            const int iq = (int)((h >> 8) & 0xffffffu);
            if (bq > bl || (bq == bl && iq < il)) { bl = bq; il = iq; wl = q; }
          }
          if (__all_sync(0xffffffffu, mine)) {
            ok = true;
            b2 = bl;
            i2 = il;
            w2 = wl;
            break;
          }
          if ((it & 31) == 31 && ld_acquire_gpu(abort_flag)) break;
          if (it > 16) __nanosleep(32);
        }
        if (!ok) {
          if (lane == 0) {
            atomicOr(err, 8);
            atomicExch(abort_flag, 1u);
            s_abort = 1;
          }
        } else {
          for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, b2, o);
            const int oi = __shfl_xor_sync(0xffffffffu, i2, o);
            const int ow = __shfl_xor_sync(0xffffffffu, w2, o);
            if (ob > b2 || (ob == b2 && oi < i2)) { b2 = ob; i2 = oi; w2 = ow; }
          }
          if (i2 >= n) i2 = c;
          if (lane == 0) {
            s_p = i2;
            s_piv[cc] = i2;
            if (j == 0) {
              piv[(int64_t)z * n + c] = i2;
              if (!(b2 > 0) && info) atomicOr(info + z, 1);
            }
          }
          if (lane < l) {
            s_u[lane] = ldcg_cx(&cb[w2].v[lane]);
            s_d[lane] = ldcg_cx(&cb[0].d[lane]);
          }
        }
      }
      __syncthreads();
      if (s_abort) return;
      const int p = s_p;
      // rows c and p exchange (row c takes the pivot row; the thread of row p, below, restores
      // the former row c into it); rows below c are scaled and updated, and each thread keeps its
      // best candidate for the next column
      if (p != c && tid < l && c >= r_lo && c < r_hi) S[tid * ch + c - r_lo] = s_u[tid];
      const Cx<float> d = s_u[cc];
      const float dd = d.re * d.re + d.im * d.im;
      const bool okd = dd > 0.f;
      best = -1.f;
      bi = n;
      for (int r = max(a, c + 1) + tid; r < r_hi; r += NT) {
        if (r == p)
          for (int t = 0; t < l; ++t) S[t * ch + r - r_lo] = s_d[t];
        Cx<float> lv = S[cc * ch + r - r_lo];
        if (okd) lv = cx_div(lv, d);
        S[cc * ch + r - r_lo] = lv;
        for (int t = cc + 1; t < l; ++t) {
          const Cx<float> u = s_u[t];
          Cx<float>& x = S[t * ch + r - r_lo];
          x.re -= lv.re * u.re - lv.im * u.im;
          x.im -= lv.re * u.im + lv.im * u.re;
          if (t == cc + 1) {
            const float m = x.re * x.re + x.im * x.im;
            if (m > best) { best = m; bi = r; }
          }
        }
      }
      // (the next column's first __syncthreads orders these updates before any read of them)
    }
    __syncthreads();
    for (int e = tid; e < nr * l; e += NT) {
      const int rr = e / l, t = e - rr * l;
      M[(int64_t)(a + rr) * ld + c0 + t] = S[t * ch + a - r_lo + rr];
    }
    if (j == 0) {
      // net effect of the leaf's interchanges on the rows they touch: row s_rows[i] receives the
      // former row s_src[i]; the leaf's own rows c0 .. c0+l-1 come first
      if (tid == 0) {
        int m = 0;
        for (int t = 0; t < l; ++t) { s_rows[m] = c0 + t; s_src[m] = c0 + t; ++m; }
        for (int t = 0; t < l; ++t) {
          const int pr = s_piv[t];
          if (pr == c0 + t) continue;
          int ip = -1;
          for (int i = 0; i < m; ++i)
            if (s_rows[i] == pr) { ip = i; break; }
          if (ip < 0) { s_rows[m] = pr; s_src[m] = pr; ip = m++; }
          const int tmp = s_src[t];
          s_src[t] = s_src[ip];
          s_src[ip] = tmp;
        }
        s_m = m;
      }
      __syncthreads();
      const int m = s_m;
      for (int jj = p0 + tid; jj < pend; jj += NT) {  // the panel's columns outside the leaf
        if (jj >= c0 && jj < c0 + l) continue;
        Cx<float> v[2 * LWMAX];
        for (int i = 0; i < m; ++i) v[i] = ldcg_cx(M + (int64_t)s_src[i] * ld + jj);
        if (jj >= c0 + l)  // U block: forward substitution with the leaf's unit lower L11
          for (int s = 1; s < l; ++s)
            for (int t = 0; t < s; ++t) {
              const Cx<float> lv = S[t * ch + c0 + s - r_lo];
              v[s].re -= lv.re * v[t].re - lv.im * v[t].im;
              v[s].im -= lv.re * v[t].im + lv.im * v[t].re;
            }
        for (int i = 0; i < m; ++i) M[(int64_t)s_rows[i] * ld + jj] = v[i];
      }
    }
    if (!barrier()) return;
    const int cs = c0 + l, wr = pend - cs;
    if (wr > 0) {  // rows below the leaf, panel columns right of it: A -= L_leaf U_leaf
      for (int e = tid; e < l * wr; e += NT) {
        const int t = e / wr, jj = e - t * wr;
        Ub[t * coop::WMAX + jj] = ldcg_cx(M + (int64_t)(c0 + t) * ld + cs + jj);
      }
      __syncthreads();
      const int rb = max(r_lo, cs);
      const int nrow = max(0, r_hi - rb);
      if ((wr & 1) == 0 && ((ld | cs) & 1) == 0 && (bstride & 1) == 0) {  // two columns per thread, 16-byte accesses
        const int hw = wr >> 1;
#pragma unroll 2
        for (int e = tid; e < nrow * hw; e += NT) {
          const int rr = e / hw, jj = 2 * (e - rr * hw), r = rb + rr;
          float4* mp = reinterpret_cast<float4*>(M + (int64_t)r * ld + cs + jj);
          float4 acc = __ldcg(mp);
          for (int t = 0; t < l; ++t) {
            const Cx<float> lv = S[t * ch + r - r_lo];
            const float4 u = *reinterpret_cast<const float4*>(Ub + t * coop::WMAX + jj);
            acc.x -= lv.re * u.x - lv.im * u.y;
            acc.y -= lv.re * u.y + lv.im * u.x;
            acc.z -= lv.re * u.z - lv.im * u.w;
            acc.w -= lv.re * u.w + lv.im * u.z;
          }
          *mp = acc;
        }
      } else {
        for (int e = tid; e < nrow * wr; e += NT) {
          const int rr = e / wr, jj = e - rr * wr, r = rb + rr;
          Cx<float>* mp = M + (int64_t)r * ld + cs + jj;
          Cx<float> acc = ldcg_cx(mp);
          for (int t = 0; t < l; ++t) {
            const Cx<float> lv = S[t * ch + r - r_lo], u = Ub[t * coop::WMAX + jj];
            acc.re -= lv.re * u.re - lv.im * u.im;
            acc.im -= lv.re * u.im + lv.im * u.re;
          }
          *mp = acc;
        }
      }
      __syncthreads();
    }
  }
}

// Leaf width for a panel whose rows start at p0: the widest power of two <= 16 whose leaf and U
// block (lw x 64) fit in 200 KB of shared memory (fewer, wider leaves re-read the panel fewer
// times); 0 if even one column does not fit (then the global-memory panel runs).
template <class S>
static int leaf_width(int n, int p0) {
  const size_t rows = (size_t)(n - p0);
  for (int lw = 16; lw >= 1; lw >>= 1)
    if ((rows + 64) * lw * sizeof(Cx<S>) <= 200 * 1024) return lw;
  return 0;
}

template <class S>
static int panel_factor(bie_ctx* c, Cx<S>* A, int batch, int n, int ld, int64_t bstride, int p0, int w,
                        int32_t* piv, int32_t* info) {
  const int lw = leaf_width<S>(n, p0);
  if (lw == 0 || w > 64) {
    BIE_LAUNCH(k_panel<S><<<batch, 512, 0, c->stream>>>(A, bstride, n, ld, p0, w, piv, info));
    return BIE_OK;
  }
  BIE_TRY((set_smem_max(k_leaf<S>)));
  // With a large batch the leaf kernel (one CTA per matrix) also updates the panel right of the
  // leaf; with a small one that update runs as its own launch over all rows of every matrix.
  const int fuse = batch >= 64 ? 1 : 0;
  for (int c0 = p0; c0 < p0 + w; c0 += lw) {
    const int l = std::min(lw, p0 + w - c0);
    const int wr = std::max(0, std::min(p0 + w, n) - c0 - l);  // panel columns right of the leaf
    const size_t smem = ((size_t)(n - c0) * l + (size_t)l * std::min(w, n - p0)) * sizeof(Cx<S>);
    BIE_LAUNCH(k_leaf<S><<<batch, 1024, smem, c->stream>>>(A, bstride, n, ld, p0, w, c0, l, piv, info, fuse));
    const int rows = n - c0 - l;
    if (!fuse && rows > 0 && wr > 0) {
      dim3 g((unsigned)((rows + 63) / 64), batch);
      BIE_LAUNCH(k_leaf_update<S><<<g, 256, 0, c->stream>>>(A, bstride, n, ld, p0, w, c0, l));
    }
  }
  return BIE_OK;
}

// ---- row swaps outside the panel, then U12 = L11^{-1} A12 ----------------------------------
// grid: (ceil((n - jlo) / 128), batch), block 128: one column j >= jlo per thread.  With swaps != 0
// the panel's row swaps are applied (in order) to every column outside the panel; the forward
// substitution with the unit lower L11 runs for the columns in [p0 + nb, tend).
template <class S>
__global__ void __launch_bounds__(128) k_swap_trsm(Cx<S>* __restrict__ A, int64_t bstride, int n, int ld, int p0,
                                                   int nb, const int32_t* __restrict__ piv, int jlo, int tend,
                                                   int swaps) {
  Cx<S>* M = A + (int64_t)blockIdx.y * bstride;
  const int32_t* pv = piv + (int64_t)blockIdx.y * n;
  extern __shared__ unsigned char smem_raw[];
  Cx<S>* L11 = reinterpret_cast<Cx<S>*>(smem_raw);  // [nb][nb]
  const int pend = min(p0 + nb, n);
  const int w = pend - p0;
  if (tend > pend) {  // some column is solved: stage L11
    for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
      int r = t / w, cc = t % w;
      L11[t] = M[(int64_t)(p0 + r) * ld + p0 + cc];
    }
    __syncthreads();
  }
  const int j = jlo + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n || (j >= p0 && j < pend)) return;
  if (swaps)
    for (int s = p0; s < pend; ++s) {
      int p = pv[s];
      if (p != s) {
        Cx<S> t = M[(int64_t)s * ld + j];
        M[(int64_t)s * ld + j] = M[(int64_t)p * ld + j];
        M[(int64_t)p * ld + j] = t;
      }
    }
  if (j < pend || j >= tend) return;  // columns left of the panel (or past tend) only get the swaps
  // forward substitution with the unit lower L11; solved entries are re-read from the column
  for (int s = 1; s < w; ++s) {
    Cx<S> v = M[(int64_t)(p0 + s) * ld + j];
    for (int t = 0; t < s; ++t) {
      const Cx<S> l = L11[s * w + t];
      const Cx<S> xt = M[(int64_t)(p0 + t) * ld + j];
      v.re -= l.re * xt.re - l.im * xt.im;
      v.im -= l.re * xt.im + l.im * xt.re;
    }
    M[(int64_t)(p0 + s) * ld + j] = v;
  }
}

// ---- U = L11^{-1} A for a full 64-row panel, FP32 --------------------------------------------
// grid (ceil((j1 - j0) / 64), batch), block 64, dynamic smem 64 KB: one column j in [j0, j1) per
// thread, solved in four blocks of 16 rows.  A block's 16 entries live in registers: first the
// products with the solved entries of the earlier blocks (a loop over t that reads x_t from this
// thread's shared-memory column and L11's column t as 16-byte broadcasts), then the solve inside
// the block (unrolled).  Each x_s receives its updates in increasing t, the order of the row-by-row
// substitution of k_swap_trsm.  (A fully unrolled 64-entry register version ran from the
// instruction cache's misses.)
// With bt.ub set, each solved column also goes, rounded to TF32, into the B^T buffer of the
// tensor-core update (the real embedding: B^T rows 2 (j - bt.cb) and 2 (j - bt.cb) + 1 get, at
// floats bt.koff + 2 s, [ur, -ui] and [ui, ur]; rows bt.krow floats long, bt.stride per matrix),
// which saves the separate build pass over U.
struct BtOut {
  float* ub;
  int64_t stride;
  int krow, koff, cb;
};
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
constexpr size_t kTrsmSmem = 2 * 64 * 64 * sizeof(Cx<float>);  // L11^T and the solved columns
__global__ void __launch_bounds__(64) k_trsm64(Cx<float>* __restrict__ A, int64_t bstride, int n, int ld, int p0,
                                               int j0, int j1, BtOut bt) {
  extern __shared__ float4 trsm_smem[];
  Cx<float>* LT = reinterpret_cast<Cx<float>*>(trsm_smem);  // LT[t * 64 + s] = L11[s][t]
  Cx<float>(*X)[64] = reinterpret_cast<Cx<float>(*)[64]>(LT + 64 * 64);  // X[s][thread]: the solved column
  Cx<float>* M = A + (int64_t)blockIdx.y * bstride;
  const int tid = threadIdx.x;
#pragma unroll 8
  for (int e = tid; e < 64 * 64; e += 64) {
    const int r = e >> 6, c = e & 63;  // coalesced read of row r
    LT[c * 64 + r] = M[(int64_t)(p0 + r) * ld + p0 + c];
  }
  __syncthreads();
  const int j = j0 + blockIdx.x * blockDim.x + tid;
  const bool act = j < j1 && j < n;
#pragma unroll 1
  for (int b0 = 0; b0 < 64; b0 += 16) {
    Cx<float> xb[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) xb[r] = act ? M[(int64_t)(p0 + b0 + r) * ld + j] : Cx<float>{0.f, 0.f};
#pragma unroll 2
    for (int t = 0; t < b0; ++t) {  // earlier blocks
      const Cx<float> xt = X[t][tid];
      const float4* l4 = reinterpret_cast<const float4*>(&LT[t * 64 + b0]);
#pragma unroll
      for (int r = 0; r < 16; r += 2) {
        const float4 l = l4[r >> 1];  // L11[b0 + r][t], L11[b0 + r + 1][t]
        xb[r].re -= l.x * xt.re - l.y * xt.im;
        xb[r].im -= l.x * xt.im + l.y * xt.re;
        xb[r + 1].re -= l.z * xt.re - l.w * xt.im;
        xb[r + 1].im -= l.z * xt.im + l.w * xt.re;
      }
    }
#pragma unroll
    for (int t = 0; t < 15; ++t) {  // inside the block
      const Cx<float> xt = xb[t];
#pragma unroll
      for (int r = t + 1; r < 16; ++r) {
        const Cx<float> l = LT[(b0 + t) * 64 + b0 + r];
        xb[r].re -= l.re * xt.re - l.im * xt.im;
        xb[r].im -= l.re * xt.im + l.im * xt.re;
      }
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      X[b0 + r][tid] = xb[r];
      if (act && (b0 + r) > 0) M[(int64_t)(p0 + b0 + r) * ld + j] = xb[r];
    }
  }
  if (bt.ub && act) {  // this thread's column is complete in X
    float* o = bt.ub + (int64_t)blockIdx.y * bt.stride + (int64_t)2 * (j - bt.cb) * bt.krow + bt.koff;
#pragma unroll 4
    for (int s2 = 0; s2 < 64; s2 += 2) {
      const Cx<float> u0 = X[s2][tid], u1 = X[s2 + 1][tid];
      const float a0 = round_tf32(u0.re), b0 = round_tf32(u0.im), a1 = round_tf32(u1.re), b1 = round_tf32(u1.im);
      *reinterpret_cast<float4*>(o + 2 * s2) = make_float4(a0, -b0, a1, -b1);
      *reinterpret_cast<float4*>(o + bt.krow + 2 * s2) = make_float4(b0, a0, b1, a1);
    }
  }
}

// ---- SIMT trailing update A22 -= L21 U12 (64 x 64 complex tile per CTA, 256 threads) ---------
template <class S>
__global__ void __launch_bounds__(256) k_gemm_update(Cx<S>* __restrict__ A, int64_t bstride, int n, int ld,
                                                     int p0, int nb) {
  Cx<S>* M = A + (int64_t)blockIdx.z * bstride;
  const int r0 = p0 + nb + blockIdx.y * 64, c0 = p0 + nb + blockIdx.x * 64;
  if (r0 >= n || c0 >= n) return;
  __shared__ Cx<S> Ls[16][64 + 1];  // [k][row]
  __shared__ Cx<S> Us[16][64 + 1];  // [k][col]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  Cx<S> acc[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) acc[a][b] = {0, 0};
  for (int k0 = p0; k0 < p0 + nb; k0 += 16) {
    for (int t = threadIdx.x; t < 16 * 64; t += 256) {
      int kk = t & 15, rr = t >> 4;
      int gr = r0 + rr, gk = k0 + kk;
      Ls[kk][rr] = (gr < n && gk < p0 + nb) ? M[(int64_t)gr * ld + gk] : Cx<S>{0, 0};
      int cc = t & 63, k2 = t >> 6;
      int gc = c0 + cc, gk2 = k0 + k2;
      Us[k2][cc] = (gc < n && gk2 < p0 + nb) ? M[(int64_t)gk2 * ld + gc] : Cx<S>{0, 0};
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      Cx<S> l[4], u[4];
      for (int a = 0; a < 4; ++a) l[a] = Ls[kk][ty + 16 * a];
      for (int b = 0; b < 4; ++b) u[b] = Us[kk][tx + 16 * b];
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          acc[a][b].re += l[a].re * u[b].re - l[a].im * u[b].im;
          acc[a][b].im += l[a].re * u[b].im + l[a].im * u[b].re;
        }
    }
    __syncthreads();
  }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      int gr = r0 + ty + 16 * a, gc = c0 + tx + 16 * b;
      if (gr < n && gc < n) {
        Cx<S>& m = M[(int64_t)gr * ld + gc];
        m.re -= acc[a][b].re;
        m.im -= acc[a][b].im;
      }
    }
}

// ---- solves with the factor: x = U^{-1} L^{-1} P b; one CTA per (matrix) -------------------
template <class S, class SB>
__global__ void __launch_bounds__(256) k_lu_solve(const Cx<S>* __restrict__ LU, int64_t bstride, int n, int ld,
                                                  const int32_t* __restrict__ piv, Cx<SB>* __restrict__ b,
                                                  int64_t bstride_b) {
  const Cx<S>* M = LU + (int64_t)blockIdx.x * bstride;
  const int32_t* pv = piv + (int64_t)blockIdx.x * n;
  Cx<SB>* x = b + (int64_t)blockIdx.x * bstride_b;
  __shared__ SB red[2][8];
  __shared__ Cx<SB> xr;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0)
    for (int s = 0; s < n; ++s) {
      int p = pv[s];
      if (p != s) { Cx<SB> t = x[s]; x[s] = x[p]; x[p] = t; }
    }
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    for (int ii = 0; ii < n; ++ii) {
      const int r = pass == 0 ? ii : n - 1 - ii;
      SB sr = 0, si = 0;
      const int lo = pass == 0 ? 0 : r + 1, hi = pass == 0 ? r : n;
      for (int cc = lo + tid; cc < hi; cc += blockDim.x) {
        Cx<S> l = M[(int64_t)r * ld + cc];
        Cx<SB> v = x[cc];
        sr += (SB)l.re * v.re - (SB)l.im * v.im;
        si += (SB)l.re * v.im + (SB)l.im * v.re;
      }
      for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
      }
      if (lane == 0) { red[0][warp] = sr; red[1][warp] = si; }
      __syncthreads();
      if (tid == 0) {
        SB tr = 0, ti = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { tr += red[0][w]; ti += red[1][w]; }
        Cx<SB> v = {x[r].re - tr, x[r].im - ti};
        if (pass == 1) {
          Cx<S> d = M[(int64_t)r * ld + r];
          Cx<SB> dd = {(SB)d.re, (SB)d.im};
          SB den = dd.re * dd.re + dd.im * dd.im;
          v = {(v.re * dd.re + v.im * dd.im) / den, (v.im * dd.re - v.re * dd.im) / den};
        }
        x[r] = v;
      }
      __syncthreads();
    }
  }
}

// ---- host drivers -----------------------------------------------------------------------------
template <class S>
int lu_factor_simt(bie_ctx* c, Cx<S>* A, int batch, int n, int ld, int64_t bstride, int32_t* piv, int32_t* info,
                   int nb) {
  if (nb > 64) nb = 64;
  for (int p0 = 0; p0 < n; p0 += nb) {
    const int w = std::min(nb, n - p0);
    BIE_TRY(panel_factor<S>(c, A, batch, n, ld, bstride, p0, w, piv, info));
    dim3 gs((unsigned)((n + 127) / 128), batch);
    BIE_LAUNCH(k_swap_trsm<S><<<gs, 128, (size_t)w * w * sizeof(Cx<S>), c->stream>>>(A, bstride, n, ld, p0, w, piv,
                                                                                     0, n, 1));
    const int rem = n - p0 - w;
    if (rem > 0) {
      dim3 gg((unsigned)((rem + 63) / 64), (unsigned)((rem + 63) / 64), batch);
      BIE_LAUNCH(k_gemm_update<S><<<gg, 256, 0, c->stream>>>(A, bstride, n, ld, p0, w));
    }
  }
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

size_t lu_coop_scratch_bytes(int batch) { return coop::scratch_bytes(batch, kCoopMaxGrid); }

// The cooperative panel (k_panel_coop) for the panel at p0 when it applies: a panel taller than
// the 16-column one-CTA leaf holds (1536 rows), at most half as many matrices as SMs, and a
// chunk of rows per CTA whose leaf of at least 4 columns fits shared memory.  *used tells whether
// it ran.  `coop` is the scratch of lu_coop_scratch_bytes(batch), err the LU's error word.
static int panel_coop32(bie_ctx* c, Cx<float>* A, int batch, int n, int ld, int64_t bstride, int p0, int w,
                        int32_t* piv, int32_t* info, void* coop, int32_t* err, bool* used) {
  *used = false;
  const int rows = n - p0;
  if (!coop || !c->lu_coop || w > coop::WMAX || rows <= 1536) return BIE_OK;
  int nsm = 0;
  BIE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
  int cpm = std::min(nsm / batch, (rows + 255) / 256);  // one CTA per SM (the leaf takes most of its memory)
  if (cpm < 2) return BIE_OK;
  const int ch = ((rows + cpm - 1) / cpm + 63) / 64 * 64;
  cpm = (rows + ch - 1) / ch;
  if (cpm < 2 || batch * cpm > kCoopMaxGrid) return BIE_OK;
  BIE_TRY((set_smem_max(k_panel_coop)));
  cudaFuncAttributes fa;
  BIE_CUDA_TRY(cudaFuncGetAttributes(&fa, (const void*)k_panel_coop));
  const size_t limit = (size_t)smem_optin() - fa.sharedSizeBytes;
  int lw = coop::LWMAX;
  auto smem_of = [&](int l) { return ((size_t)l * ch + (size_t)coop::LWMAX * coop::WMAX) * sizeof(Cx<float>); };
  while (lw >= 4 && smem_of(lw) > limit) lw >>= 1;
  if (lw < 4) return BIE_OK;
  lw = std::min(lw, w);
  const size_t smem = smem_of(lw);
  int per_sm = 0;
  BIE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_panel_coop, coop::NT, smem));
  if ((int64_t)per_sm * nsm < (int64_t)batch * cpm) return BIE_OK;
  char* base = (char*)coop + 256;
  unsigned* bar = (unsigned*)base;  // [batch] counters, then the abort flag
  unsigned* abort_flag = bar + batch;
  const size_t cand_off = ((size_t)(batch + 1) * 4 + 255) & ~(size_t)255;
  coop::Cand* cand = (coop::Cand*)(base + cand_off);
  BIE_CUDA_TRY(cudaMemsetAsync(bar, 0, cand_off + 2 * (size_t)batch * cpm * sizeof(coop::Cand), c->stream));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(batch * cpm));
  cfg.blockDim = dim3(coop::NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  count_launch();
  BIE_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_panel_coop, A, bstride, n, ld, p0, w, lw, cpm, ch, piv, info, bar,
                                  abort_flag, cand, err));
  *used = true;
  return BIE_OK;
}

// Panel factorisation plus row swaps (all columns) and the U12 solve of the columns in
// [p0 + w, tend) for one block column (FP32); the trailing update is left to the caller (the
// tensor-core kernels of lu_tc.cu).  coop / err: scratch and error word of the cooperative panel
// (NULL: one CTA per matrix always).
int lu_panel_steps32(bie_ctx* c, cf* A, int batch, int n, int ld, int64_t bstride, int p0, int w, int32_t* piv,
                     int32_t* info, int tend, void* coop, int32_t* err, float* ub, int64_t ub_stride, int krow,
                     int koff, bool* emitted) {
  if (emitted) *emitted = false;
  Cx<float>* M = reinterpret_cast<Cx<float>*>(A);
  bool used = false;
  BIE_TRY(panel_coop32(c, M, batch, n, ld, bstride, p0, w, piv, info, coop, err, &used));
  if (!used) BIE_TRY(panel_factor<float>(c, M, batch, n, ld, bstride, p0, w, piv, info));
  dim3 gs((unsigned)((n + 127) / 128), batch);
  if (w == 64) {  // swaps here, the solve with the register-resident kernel
    BIE_LAUNCH(k_swap_trsm<float><<<gs, 128, 0, c->stream>>>(M, bstride, n, ld, p0, w, piv, 0, p0 + w, 1));
    if (tend > p0 + w) {
      BIE_TRY((set_smem_max(k_trsm64)));
      dim3 gt((unsigned)((tend - p0 - w + 63) / 64), batch);
      const BtOut bt{ub, ub_stride, krow, koff, p0 + w};
      BIE_LAUNCH(k_trsm64<<<gt, 64, kTrsmSmem, c->stream>>>(M, bstride, n, ld, p0, p0 + w, tend, bt));
      if (emitted) *emitted = ub != nullptr;
    }
  } else {
    BIE_LAUNCH(k_swap_trsm<float><<<gs, 128, (size_t)w * w * sizeof(Cx<float>), c->stream>>>(M, bstride, n, ld, p0, w,
                                                                                            piv, 0, tend, 1));
  }
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

// U = L11^{-1} A for rows [p0, p0 + w) and the columns [jlo, n), L11 the unit lower diagonal block
// at (p0, p0) (FP32; no swaps).
int lu_trsm_rows32(bie_ctx* c, cf* A, int batch, int n, int ld, int64_t bstride, int p0, int w, int jlo, float* ub,
                   int64_t ub_stride, int krow, int koff, bool* emitted) {
  if (emitted) *emitted = false;
  if (jlo >= n) return BIE_OK;
  Cx<float>* M = reinterpret_cast<Cx<float>*>(A);
  dim3 gs((unsigned)((n - jlo + 127) / 128), batch);
  if (w == 64) {
    BIE_TRY((set_smem_max(k_trsm64)));
    dim3 gt((unsigned)((n - jlo + 63) / 64), batch);
    const BtOut bt{ub, ub_stride, krow, koff, jlo};
    BIE_LAUNCH(k_trsm64<<<gt, 64, kTrsmSmem, c->stream>>>(M, bstride, n, ld, p0, jlo, n, bt));
    if (emitted) *emitted = ub != nullptr;
  }
  else
    BIE_LAUNCH(k_swap_trsm<float><<<gs, 128, (size_t)w * w * sizeof(Cx<float>), c->stream>>>(M, bstride, n, ld, p0, w,
                                                                                            nullptr, jlo, n, 0));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int lu_factor64(bie_ctx* c, cd* A, int batch, int n, int ld, int64_t bstride, int32_t* piv, int32_t* info) {
  return lu_factor_simt<double>(c, reinterpret_cast<Cx<double>*>(A), batch, n, ld, bstride, piv, info, 32);
}
int lu_solve64(bie_ctx* c, const cd* LU, int batch, int n, int ld, int64_t bstride, const int32_t* piv, cd* b,
               int64_t bstride_b) {
  BIE_LAUNCH(k_lu_solve<double, double><<<batch, 256, 0, c->stream>>>(reinterpret_cast<const Cx<double>*>(LU), bstride, n, ld,
                                                           piv, reinterpret_cast<Cx<double>*>(b), bstride_b));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}
// FP32 LU without tensor cores for systems the TF32 factor cannot refine: 64-column panels
// (cooperative for a few tall matrices, see k_panel_coop), their row swaps and U blocks, and the
// trailing update A22 -= L21 U12 in FP32 on the CUDA cores (k_gemm_update).  coop / err: the
// cooperative panel's scratch and error word.
int lu_factor32_panels(bie_ctx* c, cf* A, int batch, int n, int ld, int64_t bstride, int32_t* piv, int32_t* info,
                       void* coop, int32_t* err) {
  Cx<float>* M = reinterpret_cast<Cx<float>*>(A);
  BIE_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), c->stream));
  for (int p0 = 0; p0 < n; p0 += 64) {
    const int w = std::min(64, n - p0);
    BIE_TRY(lu_panel_steps32(c, A, batch, n, ld, bstride, p0, w, piv, info, n, coop, err, nullptr, 0, 0, 0, nullptr));
    const int rem = n - p0 - w;
    if (rem > 0) {
      dim3 gg((unsigned)((rem + 63) / 64), (unsigned)((rem + 63) / 64), batch);
      BIE_LAUNCH(k_gemm_update<float><<<gg, 256, 0, c->stream>>>(M, bstride, n, ld, p0, w));
    }
  }
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int lu_factor32(bie_ctx* c, cf* A, int batch, int n, int ld, int64_t bstride, int32_t* piv, int32_t* info) {
  return lu_factor_simt<float>(c, reinterpret_cast<Cx<float>*>(A), batch, n, ld, bstride, piv, info, 32);
}
int lu_solve32(bie_ctx* c, const cf* LU, int batch, int n, int ld, int64_t bstride, const int32_t* piv, cf* b,
               int64_t bstride_b) {
  BIE_LAUNCH(k_lu_solve<float, float><<<batch, 256, 0, c->stream>>>(reinterpret_cast<const Cx<float>*>(LU), bstride, n, ld, piv,
                                                         reinterpret_cast<Cx<float>*>(b), bstride_b));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

}  // namespace bie
