// mixed.cu -- the mixed-precision frequency solves (BIE_MODE_MIXED):
//   FP32 assembly with float-float phases (asm32.cu) -> FP32 copy factored by the blocked LU
//   (trailing update on the tensor cores, lu_tc.cu, or SIMT FP32 where tcgen05 is not used) ->
//   iterative refinement against the assembled matrix with float-float residuals (refine.cu).
// Frequencies whose refinement does not converge are re-solved by the FP64 path and flagged.
#include <algorithm>

#include "bie_common.cuh"

namespace bie {

int assemble32(bie_ctx* c, const double* kv, int nk, cf* A, int64_t lda, cd* b, cd* known, double* rowsum);
int lu_factor32(bie_ctx* c, cf* A, int batch, int n, int ld, int64_t bstride, int32_t* piv, int32_t* info);
int lu_factor_tc(bie_ctx* c, cf* A, int batch, int n, int ld, int64_t bstride, int32_t* piv, int32_t* info,
                 void* scratch, size_t scratch_bytes);
size_t lu_tc_scratch_bytes(int batch, int n);
int refine_solve(bie_ctx* c, const cf* A, const cf* LU, int nk, int n, int64_t ld, int64_t bstride,
                 const int32_t* piv, const cd* b, cd* x, cd* r, double* rowabs, int32_t* perm, void* state_dev,
                 int it_max, double tol);
size_t refine_state_bytes(int nk);
int refine_read_state(bie_ctx* c, const void* state_dev, int nk, int32_t* done, int32_t* iters, double* berr,
                      double* err_est);
int solve_fp64(bie_ctx* c, const double* k, int64_t Nk, cd* surf_out, bie_report* rep);
__global__ void k_surface_fields(const uint8_t* __restrict__ bc, int64_t N, const cd* __restrict__ x,
                                 const cd* __restrict__ known, cd* __restrict__ surf);

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int solve_mixed(bie_ctx* c, const double* k, int64_t Nk, cd* surf_out, bie_report* rep) {
  const int64_t N = c->N;
  const int64_t ld = (N + 63) / 64 * 64;
  const size_t mat = align256((size_t)N * ld * sizeof(cf));
  const size_t vec = align256((size_t)N * sizeof(cd));
  const size_t perk = 2 * mat + 4 * vec + align256((size_t)N * 6 * sizeof(double)) + align256((size_t)N * 8) +
                      2 * align256((size_t)N * 4) + align256(refine_state_bytes(1)) + 64;
  size_t free_b = 0, total_b = 0;
  BIE_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  int64_t kb = std::max<int64_t>(1, std::min<int64_t>(Nk, std::min<int64_t>(c->mixed_batch, (int64_t)((free_b / 2) / perk))));
  size_t tc_scratch = lu_tc_scratch_bytes((int)kb, (int)N);
  if ((size_t)kb * perk + tc_scratch > free_b)
    return fail(BIE_ERR_OOM, "mixed-precision workspace for N = " + std::to_string(N) + " does not fit");
  BIE_TRY(ensure_buf(c->work, kb * perk + tc_scratch + 8192));
  char* p = (char*)c->work.p;
  auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return (void*)q; };
  cf* A = (cf*)take(kb * mat);
  cf* LU = (cf*)take(kb * mat);
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
  double* kdev = (double*)take((size_t)kb * 8);
  void* tcs = take(tc_scratch);
  const int64_t bstride = (int64_t)(mat / sizeof(cf));
  std::vector<int32_t> done(kb), iters(kb), hinfo(kb);
  std::vector<double> berr(kb), est(kb);
  std::vector<double> fallback;
  std::vector<int64_t> fallback_idx;
  for (int64_t k0 = 0; k0 < Nk; k0 += kb) {
    const int nk = (int)std::min<int64_t>(kb, Nk - k0);
    BIE_CUDA_TRY(cudaMemcpyAsync(kdev, k + k0, nk * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    BIE_CUDA_TRY(cudaMemsetAsync(info, 0, nk * sizeof(int32_t), c->stream));
    BIE_TRY(assemble32(c, kdev, nk, A, ld, b, known, rowsum));
    BIE_CUDA_TRY(cudaMemcpyAsync(LU, A, (size_t)nk * mat, cudaMemcpyDeviceToDevice, c->stream));
    if (c->use_tcgen05)
      BIE_TRY(lu_factor_tc(c, LU, nk, (int)N, (int)ld, bstride, piv, info, tcs, tc_scratch));
    else
      BIE_TRY(lu_factor32(c, LU, nk, (int)N, (int)ld, bstride, piv, info));
    BIE_TRY(refine_solve(c, A, LU, nk, (int)N, ld, bstride, piv, b, x, r, rowabs, perm, state, c->refine_it_max,
                         c->refine_tol));
    dim3 g((unsigned)((N + 255) / 256), nk);
    k_surface_fields<<<g, 256, 0, c->stream>>>(c->bc, N, x, known, surf_out + k0 * 2 * N);
    BIE_CUDA_TRY(cudaGetLastError());
    BIE_TRY(refine_read_state(c, state, nk, done.data(), iters.data(), berr.data(), est.data()));
    BIE_CUDA_TRY(cudaMemcpy(hinfo.data(), info, nk * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (int i = 0; i < nk; ++i) {
      const bool conv = done[i] && !hinfo[i] && std::isfinite(berr[i]);
      const bool sensitive = !(est[i] <= c->fallback_err_est);
      const bool ok = conv && !sensitive;
      if (rep)
        rep[k0 + i] = bie_report{iters[i], BIE_MODE_MIXED,
                                 (conv ? 0u : BIE_FLAG_NOT_CONVERGED) | (hinfo[i] ? BIE_FLAG_ZERO_PIVOT : 0u) |
                                     (sensitive ? BIE_FLAG_ILL_CONDITIONED : 0u),
                                 0, berr[i], est[i]};
      if (!ok) {
        fallback.push_back(k[k0 + i]);
        fallback_idx.push_back(k0 + i);
      }
    }
  }
  // frequencies the mixed path could not settle (near an interior resonance, zero pivot): FP64
  for (size_t f = 0; f < fallback.size(); ++f) {
    bie_report r64;
    BIE_TRY(solve_fp64(c, &fallback[f], 1, surf_out + fallback_idx[f] * 2 * N, &r64));
    if (rep) {
      rep[fallback_idx[f]].flags |= BIE_FLAG_FALLBACK_FP64;
      rep[fallback_idx[f]].path = BIE_MODE_FP64;
    }
  }
  return BIE_OK;
}

}  // namespace bie
