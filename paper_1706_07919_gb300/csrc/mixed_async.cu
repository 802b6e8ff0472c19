// mixed_async.cu -- the mixed-precision frequency solves of mixed.cu, stream-ordered
// (bie_solve_frequencies_async): the call returns once its work is enqueued on the context's
// stream.  The decisions that mixed.cu takes on the host between batches move to the device:
//   * a kernel turns each batch's refinement state into its reports and an ordered list of the
//     flagged wavenumbers (refinement not converged, or the FP32 assembly's estimated effect on
//     the solution above "mixed.fallback_err_est");
//   * the flagged systems are re-assembled in FP64 (float-float bulk pairs) and refined against
//     that system with their own TF32 factor in rounds of G slots, ceil(batch / G) rounds per
//     batch; a slot past the batch's count carries the wavenumber -1, which every FP64 assembly
//     kernel skips, and a converged refinement state, which every refinement kernel skips;
//   * the reports reach the caller's host array through a pinned staging copy and a host
//     function at the end of the stream's work.
// Unlike the synchronous call there is no last-resort full FP64 solve: a wavenumber whose FP64
// re-assembly still does not converge (or whose factor met a zero pivot) keeps
// BIE_FLAG_NOT_CONVERGED in its report.
#include <cstring>

#include "bie_common.cuh"

namespace bie {

int assemble32(bie_ctx* c, const double* kv, int nk, cf* A, int64_t lda, cd* b, cd* known, double* rowsum, cf* kq);
int assemble64(bie_ctx* c, const double* kv, int nk, cd* A, cd* b, void* scratch, bool ff_bulk);
int lu_factor32(bie_ctx* c, cf* A, int batch, int n, int ld, int64_t bstride, int32_t* piv, int32_t* info);
int lu_factor_tc(bie_ctx* c, cf* A, int batch, int n, int ld, int64_t bstride, int32_t* piv, int32_t* info,
                 void* scratch, size_t scratch_bytes);
size_t lu_tc_scratch_bytes(int batch, int n, int block);
int lu_block_for(const bie_ctx* c, int n);
int refine_solve(bie_ctx* c, const cf* A, const cf* LU, int nk, int n, int64_t ld, int64_t bstride,
                 const int32_t* piv, const cd* b, cd* x, cd* r, double* rowabs, int32_t* perm, void* state_dev,
                 int it_max, double tol, cf* D, void* tscratch);
int64_t diag_inv_stride(int n);
int refine_fp64_system(bie_ctx* c, const cd* A64, const cd* b64, const cf* LU, int64_t ld, int64_t bstride,
                       const int32_t* perm, const int32_t* sel_dev, int ng, int n, cd* x, cd* xg, cd* r,
                       double* rowabs, void* state_dev, int it_max, double tol, const cf* D, void* tscratch,
                       bool reset_state);
size_t refine_state_bytes(int nk);
__global__ void k_surface_fields(const uint8_t* __restrict__ bc, int64_t N, const cd* __restrict__ x,
                                 const cd* __restrict__ known, cd* __restrict__ surf, int64_t kstride);

static inline size_t align256a(size_t x) { return (x + 255) & ~(size_t)255; }

// Host values reach the device as kernel parameters (copied when the launch is enqueued), so the
// caller's array is free on return without a pageable copy that may synchronise.
constexpr int kParamVals = 256;
struct ParamVals {
  double v[kParamVals];
};
__global__ void k_put_values(ParamVals pv, int n, double* __restrict__ dst) {
  if ((int)threadIdx.x < n) dst[threadIdx.x] = pv.v[threadIdx.x];
}

// Reports of a batch's nk systems (rep [nk]) and, in order, the indices of the flagged ones
// (list [nk], *count).  lu_err: the factorisation's error word (a bounded wait that gave up voids
// every factor of the batch: all reported NOT_CONVERGED, none re-assembled), or null.  One CTA.
__global__ void k_async_reports(const RefineState* __restrict__ st, const int32_t* __restrict__ info,
                                const int32_t* __restrict__ lu_err, int nk, double thresh,
                                bie_report* __restrict__ rep, int32_t* __restrict__ list,
                                int32_t* __restrict__ count) {
  const bool void_factor = lu_err && *lu_err;
  for (int i = threadIdx.x; i < nk; i += blockDim.x) {
    const bool conv = st[i].done && isfinite(st[i].berr);
    const bool sensitive = !(st[i].err_est <= thresh);
    bie_report r;
    r.iters = st[i].iters;
    r.path = BIE_MODE_MIXED;
    r.flags = (conv ? 0u : BIE_FLAG_NOT_CONVERGED) | (info[i] ? BIE_FLAG_ZERO_PIVOT : 0u) |
              (sensitive ? BIE_FLAG_ILL_CONDITIONED : 0u);
    if (info[i] || void_factor) r.flags |= BIE_FLAG_NOT_CONVERGED;  // nothing to refine with
    r.reserved = 0;
    r.backward_err = void_factor ? (double)NAN : st[i].berr;
    r.err_est = st[i].err_est;
    rep[i] = r;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0;
    for (int i = 0; i < nk; ++i) {
      const bool conv = st[i].done && isfinite(st[i].berr);
      const bool sensitive = !(st[i].err_est <= thresh);
      if (!info[i] && !void_factor && (!conv || sensitive)) list[n++] = i;
    }
    *count = n;
  }
}

// Slots of round r: slot g takes the flagged system list[r G + g] while there is one, else it is
// idle (selection -1, wavenumber -1, refinement state converged).  One CTA of >= G threads.
__global__ void k_async_round(const int32_t* __restrict__ list, const int32_t* __restrict__ count, int r, int G,
                              const double* __restrict__ kdev, double* __restrict__ kg, int32_t* __restrict__ sel,
                              RefineState* __restrict__ stg) {
  const int g = threadIdx.x;
  if (g >= G) return;
  const int idx = r * G + g;
  const bool active = idx < *count;
  sel[g] = active ? list[idx] : -1;
  kg[g] = active ? kdev[list[idx]] : -1.0;
  RefineState s;
  memset(&s, 0, sizeof(s));
  s.done = active ? 0 : 1;
  stg[g] = s;
}

// Reports of the round's active slots after their FP64 refinement.
__global__ void k_async_round_reports(const int32_t* __restrict__ sel, const RefineState* __restrict__ stg, int G,
                                      bie_report* __restrict__ rep) {
  const int g = threadIdx.x;
  if (g >= G || sel[g] < 0) return;
  bie_report& r = rep[sel[g]];
  r.flags |= BIE_FLAG_FP64_ASSEMBLY;
  r.iters += stg[g].iters;
  r.backward_err = stg[g].berr;
  if (stg[g].done && isfinite(stg[g].berr))
    r.flags &= ~BIE_FLAG_NOT_CONVERGED;
  else
    r.flags |= BIE_FLAG_NOT_CONVERGED;
}

namespace {
struct HostCopy {
  void* dst;
  const void* src;
  size_t bytes;
};
void CUDART_CB host_copy(void* p) {
  HostCopy* h = static_cast<HostCopy*>(p);
  std::memcpy(h->dst, h->src, h->bytes);
  delete h;
}
}  // namespace

constexpr int kAsyncGroupMax = 32;  // FP64 re-assembly slots per round (at most)

int solve_mixed_async(bie_ctx* c, const double* k, int64_t Nk, cd* surf_out, bie_report* rep) {
  const int64_t N = c->N;
  const int64_t ld = (N + 63) / 64 * 64;
  const size_t mat = align256a((size_t)N * ld * sizeof(cf));
  const size_t vec = align256a((size_t)N * sizeof(cd));
  const int64_t dstride = diag_inv_stride((int)N);
  const size_t dsz = align256a((size_t)dstride * sizeof(cf));
  const size_t perk = 2 * mat + dsz + 4 * vec + align256a((size_t)N * 6 * sizeof(double)) + align256a((size_t)N * 8) +
                      2 * align256a((size_t)N * 4) + align256a(refine_state_bytes(1)) + 64 +
                      align256a(sizeof(bie_report)) + 16;
  const size_t fb1 = align256a((size_t)N * N * sizeof(cd)) + 7 * vec + align256a((size_t)N * 8) + 1024;
  if (rep && c->rep_pinned_bytes < (size_t)Nk * sizeof(bie_report)) {
    // report staging, grown before this call enqueues anything; a smaller earlier buffer is
    // retired, not freed, since an earlier call's host function may still read it (freed with
    // the context)
    if (c->rep_pinned) c->rep_pinned_old.push_back(c->rep_pinned);
    c->rep_pinned = nullptr;
    c->rep_pinned_bytes = 0;
    const size_t want = std::max<size_t>((size_t)Nk * sizeof(bie_report), 4096);
    BIE_CUDA_TRY(cudaMallocHost(&c->rep_pinned, want));
    c->rep_pinned_bytes = want;
  }
  size_t free_b = 0;
  BIE_TRY(device_free(c, &free_b));
  const int G = (int)std::max<size_t>(
      1, std::min<size_t>(std::min(kAsyncGroupMax, c->reassembly_group), (free_b / 8) / fb1));
  const size_t fb = (size_t)G * fb1 + 4096;
  const size_t avail = free_b > fb ? free_b - fb : 0;
  int64_t kb = std::max<int64_t>(1, std::min<int64_t>(Nk, std::min<int64_t>(c->mixed_batch, (int64_t)((avail / 2) / perk))));
  const size_t fixed = align256a((size_t)Nk * sizeof(double)) + align256a((size_t)Nk * sizeof(bie_report)) + 4096;
  size_t tc_scratch = lu_tc_scratch_bytes((int)kb, (int)N, lu_block_for(c, (int)N));
  if ((size_t)kb * perk + tc_scratch + fb + fixed > free_b)
    return fail(BIE_ERR_OOM, "mixed-precision workspace for N = " + std::to_string(N) + " does not fit");
  for (;;) {
    const int rc = ensure_buf(c, c->work, kb * perk + tc_scratch + fb + fixed + 16384);
    if (rc == BIE_OK) break;
    if (rc != BIE_ERR_OOM || kb == 1) return rc;
    kb = std::max<int64_t>(1, kb / 2);
    tc_scratch = lu_tc_scratch_bytes((int)kb, (int)N, lu_block_for(c, (int)N));
  }
  char* p = (char*)c->work.p;
  auto take = [&](size_t bytes) { char* q = p; p += align256a(bytes); return (void*)q; };
  cf* A = (cf*)take(kb * mat);
  cf* LU = (cf*)take(kb * mat);
  cf* Dinv = (cf*)take(kb * dsz);
  cd* b = (cd*)take(kb * vec);
  cd* x = (cd*)take(kb * vec);
  cd* r = (cd*)take(kb * vec);
  cd* known = (cd*)take(kb * vec);
  double* rowsum = (double*)take((size_t)kb * N * 6 * sizeof(double));
  double* rowabs = (double*)take((size_t)kb * N * sizeof(double));
  int32_t* piv = (int32_t*)take((size_t)kb * N * 4);
  int32_t* perm = (int32_t*)take((size_t)kb * N * 4);
  void* state = take(refine_state_bytes((int)kb));
  int32_t* info = (int32_t*)take((size_t)kb * 4);
  int32_t* list = (int32_t*)take((size_t)kb * 4);
  int32_t* count = (int32_t*)take(256);
  void* tcs = take(tc_scratch);
  cd* A64 = (cd*)take((size_t)G * N * N * sizeof(cd));
  cd* b64 = (cd*)take((size_t)G * vec);
  cd* s64 = (cd*)take((size_t)G * 4 * vec);
  cd* xg = (cd*)take((size_t)G * vec);
  cd* rg = (cd*)take((size_t)G * vec);
  double* rowabs_g = (double*)take((size_t)G * N * sizeof(double));
  void* state_g = take(refine_state_bytes(G));
  double* kg = (double*)take(G * sizeof(double));
  int32_t* sel_g = (int32_t*)take(G * sizeof(int32_t));
  double* kall = (double*)take((size_t)Nk * sizeof(double));
  bie_report* rep_dev = (bie_report*)take((size_t)Nk * sizeof(bie_report));
  const int64_t bstride = (int64_t)(mat / sizeof(cf));
  for (int64_t i0 = 0; i0 < Nk; i0 += kParamVals) {
    ParamVals pv;
    const int n = (int)std::min<int64_t>(kParamVals, Nk - i0);
    for (int i = 0; i < n; ++i) pv.v[i] = k[i0 + i];
    BIE_LAUNCH(k_put_values<<<1, kParamVals, 0, c->stream>>>(pv, n, kall + i0));
  }
  const int rounds_per_batch = (int)((kb + G - 1) / G);
  for (int64_t k0 = 0; k0 < Nk; k0 += kb) {
    const int nk = (int)std::min<int64_t>(kb, Nk - k0);
    const double* kdev = kall + k0;
    BIE_CUDA_TRY(cudaMemsetAsync(info, 0, nk * sizeof(int32_t), c->stream));
    BIE_TRY(assemble32(c, kdev, nk, A, ld, b, known, rowsum, LU));  // LU is free until the copy below
    BIE_CUDA_TRY(cudaMemcpyAsync(LU, A, (size_t)nk * mat, cudaMemcpyDeviceToDevice, c->stream));
    if (c->tc_version > 0)
      BIE_TRY(lu_factor_tc(c, LU, nk, (int)N, (int)ld, bstride, piv, info, tcs, tc_scratch));
    else
      BIE_TRY(lu_factor32(c, LU, nk, (int)N, (int)ld, bstride, piv, info));
    BIE_TRY(refine_solve(c, A, LU, nk, (int)N, ld, bstride, piv, b, x, r, rowabs, perm, state, c->refine_it_max,
                         c->refine_tol, Dinv, rowsum));
    BIE_LAUNCH(k_async_reports<<<1, 256, 0, c->stream>>>((const RefineState*)state, info,
                                                         c->tc_version > 0 ? (const int32_t*)tcs : nullptr, nk,
                                                         c->fallback_err_est, rep_dev + k0, list, count));
    const int rounds = std::min(rounds_per_batch, (nk + G - 1) / G);
    for (int rr = 0; rr < rounds; ++rr) {
      BIE_LAUNCH(k_async_round<<<1, ((G + 31) / 32) * 32, 0, c->stream>>>(list, count, rr, G, kdev, kg, sel_g,
                                                                         (RefineState*)state_g));
      BIE_TRY(assemble64(c, kg, G, A64, b64, s64, c->reassembly_ff != 0));
      BIE_TRY(refine_fp64_system(c, A64, b64, LU, ld, bstride, perm, sel_g, G, (int)N, x, xg, rg, rowabs_g, state_g,
                                 c->refine64_it_max, c->refine64_tol, Dinv, s64, false));
      BIE_LAUNCH(k_async_round_reports<<<1, ((G + 31) / 32) * 32, 0, c->stream>>>(sel_g, (const RefineState*)state_g,
                                                                                G, rep_dev + k0));
    }
    dim3 g((unsigned)((N + 255) / 256), nk);
    BIE_LAUNCH(k_surface_fields<<<g, 256, 0, c->stream>>>(c->bc, N, x, known, surf_out + k0 * 2 * N, 2 * N));
    BIE_CUDA_TRY(cudaGetLastError());
  }
  if (rep) {  // reports: device -> pinned staging -> the caller's array, in stream order
    const size_t bytes = (size_t)Nk * sizeof(bie_report);
    BIE_CUDA_TRY(cudaMemcpyAsync(c->rep_pinned, rep_dev, bytes, cudaMemcpyDeviceToHost, c->stream));
    HostCopy* h = new HostCopy{rep, c->rep_pinned, bytes};
    const cudaError_t e = cudaLaunchHostFunc(c->stream, host_copy, h);
    if (e != cudaSuccess) {
      delete h;
      return cuda_fail(e, "cudaLaunchHostFunc");
    }
  }
  return BIE_OK;
}

}  // namespace bie
