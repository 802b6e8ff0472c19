// mixed.cu -- the mixed-precision frequency solves (BIE_MODE_MIXED):
//   FP32 assembly with float-float phases (asm32.cu) -> FP32 copy factored by the blocked LU
//   (trailing update on the tcgen05 tensor cores, lu_tc.cu, or SIMT FP32) -> iterative refinement
//   against the assembled matrix with float-float residuals (refine.cu).
// Wavenumbers whose estimated sensitivity to the FP32 assembly is too high (next to an interior
// resonance) or whose refinement stalled are re-assembled in FP64 and refined against that system
// with the same low-precision factor; only if that also stalls does the full FP64 path run.
#include <algorithm>

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
size_t trsv_scratch_bytes(int nk, int n);
int lu_tc_error(bie_ctx* c, void* scratch, int32_t* out);
int lu_factor32_panels(bie_ctx* c, cf* A, int batch, int n, int ld, int64_t bstride, int32_t* piv, int32_t* info,
                       void* coop, int32_t* err);
int factor_aux(bie_ctx* c, const cf* LU, int nk, int n, int64_t ld, int64_t bstride, const int32_t* piv,
               int32_t* perm, cf* D);
int64_t diag_inv_stride(int n);
int refine_fp64_system(bie_ctx* c, const cd* A64, const cd* b64, const cf* LU, int64_t ld, int64_t bstride,
                       const int32_t* perm, const int32_t* sel_dev, int ng, int n, cd* x, cd* xg, cd* r,
                       double* rowabs, void* state_dev, int it_max, double tol, const cf* D, void* tscratch,
                       bool reset_state);
size_t refine_state_bytes(int nk);
int refine_read_state(bie_ctx* c, const void* state_dev, int nk, int32_t* done, int32_t* iters, double* berr,
                      double* err_est);
int solve_fp64(bie_ctx* c, const double* k, int64_t Nk, cd* surf_out, bie_report* rep);
int rhs_from_known(bie_ctx* c, const cf* B, int nk, int n, int64_t ld, int64_t bstride, const cd* known, cd* zero,
                   cd* b, double* rowabs, void* state_dev);
int flipped_bc(bie_ctx* c, uint8_t** out);
__global__ void k_known64(const double* __restrict__ nodes, const double* __restrict__ normals,
                          const uint8_t* __restrict__ bc, int64_t N, const double* __restrict__ kv, double dx,
                          double dy, double dz, cd* __restrict__ known);
__global__ void k_surface_fields(const uint8_t* __restrict__ bc, int64_t N, const cd* __restrict__ x,
                                 const cd* __restrict__ known, cd* __restrict__ surf, int64_t kstride);

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int kFallbackGroupMax = 32;  // FP64 systems re-assembled and refined together (at most)
constexpr int kRefactorItMax = 30;     // corrections with the FP32 re-factorisation

// FP64 matrix [n][n] rounded into an FP32 one [n][ld]; grid (ceil(n / 256), n)
__global__ void k_cd_to_cf(const cd* __restrict__ A, int64_t n, cf* __restrict__ F, int64_t ld) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= n) return;
  const cd v = A[i * n + j];
  F[i * ld + j] = {(float)v.re, (float)v.im};
}

// lu_keep / perm_keep / d_keep (optional, device): receive the low-precision factor ([Nk][N][ld],
// ld = N rounded up to 64), row permutation ([Nk][N]) and diagonal-block inverses
// ([Nk][diag_inv_stride(N)]) of every wavenumber.
// dirs (host [ndir][3], unit vectors; NULL: the context's direction, ndir = 1): several incident
// plane waves share each wavenumber's matrix and factor (Sec. 5: the solution matrix is kept and
// only the incident wave changes).  Their right-hand sides come from the known-column matrix B --
// the coefficients of the known boundary values in Eq. (BRIEF), which is the system matrix with
// every node's condition exchanged, assembled once per wavenumber by the same kernels -- as
// b_d = -B known_d (float-float products).  surf_out [Nk][ndir][2][N], rep [Nk][ndir].
int solve_mixed(bie_ctx* c, const double* k, int64_t Nk, cd* surf_out, bie_report* rep, cf* lu_keep,
                int32_t* perm_keep, cf* d_keep, const double* dirs, int ndir) {
  const int64_t N = c->N;
  if (!dirs || ndir < 1) ndir = 1;
  const bool multi = ndir > 1;
  double dir0[3] = {c->dir[0], c->dir[1], c->dir[2]};
  std::vector<double> hdirs(3 * ndir);
  for (int d = 0; d < ndir; ++d)
    for (int t = 0; t < 3; ++t) hdirs[3 * d + t] = dirs ? dirs[3 * d + t] : dir0[t];
  struct DirGuard {  // the context's direction is switched per direction and restored on return
    bie_ctx* c;
    double d[3];
    ~DirGuard() { for (int t = 0; t < 3; ++t) c->dir[t] = d[t]; }
  } dirguard{c, {dir0[0], dir0[1], dir0[2]}};
  auto set_dir = [&](int d) { for (int t = 0; t < 3; ++t) c->dir[t] = hdirs[3 * d + t]; };
  set_dir(0);
  uint8_t* bc_flip = nullptr;
  if (multi) BIE_TRY(flipped_bc(c, &bc_flip));
  const int64_t kstride = (int64_t)ndir * 2 * N;  // surf_out elements between wavenumbers
  const int64_t ld = (N + 63) / 64 * 64;
  const size_t mat = align256((size_t)N * ld * sizeof(cf));  // == N * ld * 8: ld is a multiple of 64
  const size_t vec = align256((size_t)N * sizeof(cd));
  const int64_t dstride = diag_inv_stride((int)N);
  const size_t dsz = align256((size_t)dstride * sizeof(cf));
  const size_t perk = (multi ? 3 : 2) * mat + dsz + 4 * vec + align256((size_t)N * 6 * sizeof(double)) +
                      align256((size_t)N * 8) + 2 * align256((size_t)N * 4) + align256(refine_state_bytes(1)) + 64;
  // FP64 re-assembly group: A64, b64, known/rowsum scratch, xg, r, rowabs, state, k, sel.  One
  // group refines its systems in the same launches (one CTA per system in the triangular
  // solves), so a larger group fills more of the GPU; it is capped at an eighth of free memory.
  // With one direction the flagged systems of all batches are pooled (their factor, permutation,
  // diagonal-block inverses, solution and known values copied aside) and re-assembled and refined
  // together when the pool is full and after the last batch, instead of batch by batch.
  const size_t pool1 = multi ? 0 : mat + align256((size_t)N * 4) + dsz + 2 * vec;
  const size_t fb1 = align256((size_t)N * N * sizeof(cd)) + 7 * vec + align256((size_t)N * 8) + 1024 + pool1;
  size_t free_b = 0;
  BIE_TRY(device_free(c, &free_b));
  const int G = (int)std::max<size_t>(
      1, std::min<size_t>(std::min(kFallbackGroupMax, c->reassembly_group), (free_b / 8) / fb1));
  const size_t fb = (size_t)G * fb1 + 4096;
  const size_t avail = free_b > fb ? free_b - fb : 0;
  int64_t kb = std::max<int64_t>(1, std::min<int64_t>(Nk, std::min<int64_t>(c->mixed_batch, (int64_t)((avail / 2) / perk))));
  size_t tc_scratch = lu_tc_scratch_bytes((int)kb, (int)N, lu_block_for(c, (int)N));
  if ((size_t)kb * perk + tc_scratch + fb > free_b)
    return fail(BIE_ERR_OOM, "mixed-precision workspace for N = " + std::to_string(N) + " does not fit");
  // memory shared with other contexts (scheduler workers on other streams) can run short between
  // the query above and the allocation: halve the batch and try again
  for (;;) {
    const int rc = ensure_buf(c, c->work, kb * perk + tc_scratch + fb + 16384);
    if (rc == BIE_OK) break;
    if (rc != BIE_ERR_OOM || kb == 1) return rc;
    kb = std::max<int64_t>(1, kb / 2);
    tc_scratch = lu_tc_scratch_bytes((int)kb, (int)N, lu_block_for(c, (int)N));
  }
  char* p = (char*)c->work.p;
  auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return (void*)q; };
  cf* A = (cf*)take(kb * mat);
  cf* LU = (cf*)take(kb * mat);
  cf* Bk = multi ? (cf*)take(kb * mat) : nullptr;  // known-column matrices
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
  double* kdev = (double*)take((size_t)kb * 8);
  void* tcs = take(tc_scratch);
  cd* A64 = (cd*)take((size_t)G * N * N * sizeof(cd));
  cd* b64 = (cd*)take((size_t)G * vec);
  cd* s64 = (cd*)take((size_t)G * 4 * vec);  // known + rowsum of the FP64 assembly
  cd* xg = (cd*)take((size_t)G * vec);
  cd* rg = (cd*)take((size_t)G * vec);
  double* rowabs_g = (double*)take((size_t)G * N * sizeof(double));
  void* state_g = take(refine_state_bytes(G));
  double* kg = (double*)take(G * sizeof(double));
  int32_t* sel_g = (int32_t*)take(G * sizeof(int32_t));
  cf* pLU = multi ? nullptr : (cf*)take((size_t)G * mat);  // the pool (one direction)
  int32_t* pperm = multi ? nullptr : (int32_t*)take((size_t)G * N * 4);
  cf* pD = multi ? nullptr : (cf*)take((size_t)G * dsz);
  cd* px = multi ? nullptr : (cd*)take((size_t)G * vec);
  cd* pknown = multi ? nullptr : (cd*)take((size_t)G * vec);
  std::vector<double> pool_k;
  std::vector<int64_t> pool_idx;
  const int64_t bstride = (int64_t)(mat / sizeof(cf));
  std::vector<int32_t> done(kb), iters(kb), hinfo(kb);
  std::vector<double> berr(kb), est(kb);
  std::vector<int32_t> gd(G), gi(G);
  std::vector<double> gb(G), ge(G);
  std::vector<double> full64;
  std::vector<int64_t> full64_idx;
  std::vector<int> full64_dir;
  // The device part of a batch (assembly, factorisation, refinement) is stream-ordered and needs
  // no host decision, so full batches after the first are captured once in a CUDA graph and
  // replayed; the wavenumbers reach the graph through a pinned host buffer.
  // Phase timing (option "mixed.phase_timing"): events around assembly, factorisation, refinement
  // and the re-assembly of flagged wavenumbers, read after each batch; graphs are then not used.
  const bool timing = c->phase_timing != 0;
  cudaEvent_t ev[6] = {};
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() { for (int i = 0; i < 6; ++i) if (e[i]) cudaEventDestroy(e[i]); }
  } evguard{ev};
  if (timing) {
    c->phase = bie_phase_times{};
    for (int i = 0; i < 6; ++i) BIE_CUDA_TRY(cudaEventCreate(&ev[i]));
  }
  auto mark = [&](int i) -> int {
    if (timing) BIE_CUDA_TRY(cudaEventRecord(ev[i], c->stream));
    return BIE_OK;
  };
  auto batch_core = [&](const double* ksrc, int nk) -> int {
    BIE_TRY(mark(0));
    BIE_CUDA_TRY(cudaMemcpyAsync(kdev, ksrc, nk * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    BIE_CUDA_TRY(cudaMemsetAsync(info, 0, nk * sizeof(int32_t), c->stream));
    BIE_TRY(assemble32(c, kdev, nk, A, ld, b, known, rowsum, LU));  // LU is free until the copy below
    BIE_CUDA_TRY(cudaMemcpyAsync(LU, A, (size_t)nk * mat, cudaMemcpyDeviceToDevice, c->stream));
    BIE_TRY(mark(1));
    if (c->tc_version > 0)
      BIE_TRY(lu_factor_tc(c, LU, nk, (int)N, (int)ld, bstride, piv, info, tcs, tc_scratch));
    else
      BIE_TRY(lu_factor32(c, LU, nk, (int)N, (int)ld, bstride, piv, info));
    BIE_TRY(mark(2));
    BIE_TRY(refine_solve(c, A, LU, nk, (int)N, ld, bstride, piv, b, x, r, rowabs, perm, state, c->refine_it_max,
                         c->refine_tol, Dinv, rowsum));  // the assembly's row sums are free scratch now
    BIE_TRY(mark(3));
    return BIE_OK;
  };
  auto elapsed = [&](int a, int b2) -> double {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev[a], ev[b2]) != cudaSuccess) return 0.0;
    return (double)ms;
  };
  bool use_graph = c->mixed_graph && !timing && !multi && Nk >= 2 * kb;
  double* kpin = nullptr;
  if (use_graph) {
    BIE_TRY(ensure_pinned(c, (size_t)kb * sizeof(double)));
    kpin = (double*)c->pinned;
  }
  cudaGraphExec_t gexec = nullptr;
  int64_t gnodes = 0;
  struct ExecGuard {
    cudaGraphExec_t* e;
    ~ExecGuard() { if (*e) cudaGraphExecDestroy(*e); }
  } guard{&gexec};
  // Re-assembles the pooled systems in FP64 (float-float bulk), refines them with their TF32
  // factors and writes their surface values and reports.
  auto flush_pool = [&]() -> int {
    const int ng = (int)pool_k.size();
    if (ng == 0) return BIE_OK;
    std::vector<int32_t> ident(ng);
    for (int g = 0; g < ng; ++g) ident[g] = g;
    BIE_CUDA_TRY(cudaMemcpyAsync(kg, pool_k.data(), ng * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    BIE_CUDA_TRY(cudaMemcpyAsync(sel_g, ident.data(), ng * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    BIE_TRY(mark(4));
    BIE_TRY(assemble64(c, kg, ng, A64, b64, s64, c->reassembly_ff != 0));
    BIE_TRY(refine_fp64_system(c, A64, b64, pLU, ld, bstride, pperm, sel_g, ng, (int)N, px, xg, rg, rowabs_g, state_g,
                               c->refine64_it_max, c->refine64_tol, pD, s64, true));  // the FP64 assembly's scratch
    BIE_TRY(mark(5));
    for (int g = 0; g < ng; ++g) {
      dim3 gs((unsigned)((N + 255) / 256), 1);
      BIE_LAUNCH(k_surface_fields<<<gs, 256, 0, c->stream>>>(c->bc, N, px + (int64_t)g * N, pknown + (int64_t)g * N,
                                                            surf_out + pool_idx[g] * 2 * N, 2 * N));
    }
    BIE_CUDA_TRY(cudaGetLastError());
    BIE_TRY(refine_read_state(c, state_g, ng, gd.data(), gi.data(), gb.data(), ge.data()));
    if (timing) {
      c->phase.reassembly_ms += elapsed(4, 5);
      c->phase.reassembled += ng;
    }
    for (int g = 0; g < ng; ++g) {
      const int64_t idx = pool_idx[g];
      if (rep) {
        rep[idx].flags |= BIE_FLAG_FP64_ASSEMBLY;
        rep[idx].iters += gi[g];
        rep[idx].backward_err = gb[g];
        if (gd[g]) rep[idx].flags &= ~BIE_FLAG_NOT_CONVERGED;
      }
      if (!gd[g] || !std::isfinite(gb[g])) {
        full64.push_back(pool_k[g]);
        full64_idx.push_back(idx);
        full64_dir.push_back(0);
      }
    }
    pool_k.clear();
    pool_idx.clear();
    return BIE_OK;
  };
  for (int64_t k0 = 0; k0 < Nk; k0 += kb) {
    const int nk = (int)std::min<int64_t>(kb, Nk - k0);
    if (use_graph && k0 > 0 && nk == kb) {
      std::copy(k + k0, k + k0 + nk, kpin);  // the previous batch has completed (its state was read)
      if (!gexec) {
        const int64_t before = (int64_t)bie_kernel_launches();
        cudaGraph_t graph = nullptr;
        cudaStream_t saved = nullptr;
        int rc = capture_begin(c, &saved);
        if (rc == BIE_OK) {
          rc = batch_core(kpin, nk);
          const int re = capture_end(c, saved, &graph);
          if (rc == BIE_OK && re == BIE_OK && graph)
            rc = cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess ? BIE_OK : BIE_ERR_CUDA;
          else
            rc = BIE_ERR_CUDA;
          if (graph) cudaGraphDestroy(graph);
        }
        gnodes = (int64_t)bie_kernel_launches() - before;
        uncount_launches(gnodes);  // captured, not launched: counted per replay
        if (rc != BIE_OK) {  // capture unsupported here: run this call's batches directly
          cudaGetLastError();
          if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
          use_graph = false;
        }
      }
      if (gexec) {
        BIE_CUDA_TRY(cudaGraphLaunch(gexec, c->stream));
        count_launches(gnodes);
      } else {
        BIE_TRY(batch_core(k + k0, nk));
      }
    } else {
      if (multi) {  // the known-column matrices B first (the factor's buffer is free scratch until then)
        BIE_CUDA_TRY(cudaMemcpyAsync(kdev, k + k0, nk * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        uint8_t* bc_real = c->bc;
        c->bc = bc_flip;
        const int rc = assemble32(c, kdev, nk, Bk, ld, x, r, rowsum, LU);  // b and known: discarded
        c->bc = bc_real;
        BIE_TRY(rc);
      }
      BIE_TRY(batch_core(k + k0, nk));
    }
    if (lu_keep) {
      BIE_CUDA_TRY(cudaMemcpyAsync(lu_keep + k0 * N * ld, LU, (size_t)nk * N * ld * sizeof(cf), cudaMemcpyDeviceToDevice,
                                   c->stream));
      BIE_CUDA_TRY(cudaMemcpyAsync(perm_keep + k0 * N, perm, (size_t)nk * N * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                   c->stream));
      if (d_keep)
        BIE_CUDA_TRY(cudaMemcpyAsync(d_keep + k0 * dstride, Dinv, (size_t)nk * dstride * sizeof(cf),
                                     cudaMemcpyDeviceToDevice, c->stream));
    }
    for (int d = 0; d < ndir; ++d) {
      const int64_t r0 = (k0 * ndir + d);  // report and output slot of (k0, d); wavenumbers ndir apart
      if (d > 0) {  // next incident direction: same matrices and factors, new right-hand side
        set_dir(d);
        dim3 gk((unsigned)((N + 255) / 256), nk);
        BIE_LAUNCH(k_known64<<<gk, 256, 0, c->stream>>>(c->nodes, c->normals, c->bc, N, kdev, c->dir[0], c->dir[1],
                                                       c->dir[2], known));
        BIE_TRY(rhs_from_known(c, Bk, nk, (int)N, ld, bstride, known, r, b, rowabs, state));
        BIE_TRY(refine_solve(c, A, LU, nk, (int)N, ld, bstride, piv, b, x, r, rowabs, perm, state, c->refine_it_max,
                             c->refine_tol, Dinv, rowsum));
      }
      BIE_TRY(refine_read_state(c, state, nk, done.data(), iters.data(), berr.data(), est.data()));
      if (d == 0) BIE_CUDA_TRY(cudaMemcpy(hinfo.data(), info, nk * sizeof(int32_t), cudaMemcpyDeviceToHost));
      if (d == 0 && c->tc_version > 0) {  // a bounded wait of the factorisation gave up: its factor is void
        int32_t terr = 0;
        BIE_TRY(lu_tc_error(c, tcs, &terr));
        if (terr) return fail(BIE_ERR_TIMEOUT, "LU: a bounded wait in the tensor-core update or a cooperative panel gave up");
      }
      if (timing && d == 0) {  // the batch has completed (its state was read)
        c->phase.assembly_ms += elapsed(0, 1);
        c->phase.factor_ms += elapsed(1, 2);
        c->phase.refine_ms += elapsed(2, 3);
        c->phase.batches += 1;
        c->phase.systems += nk;
      }
      std::vector<int32_t> flagged;
      for (int i = 0; i < nk; ++i) {
        const bool conv = done[i] && std::isfinite(berr[i]);
        const bool sensitive = !(est[i] <= c->fallback_err_est);
        if (rep)
          rep[r0 + (int64_t)i * ndir] = bie_report{iters[i], BIE_MODE_MIXED,
                                                   (conv ? 0u : BIE_FLAG_NOT_CONVERGED) |
                                                       (hinfo[i] ? BIE_FLAG_ZERO_PIVOT : 0u) |
                                                       (sensitive ? BIE_FLAG_ILL_CONDITIONED : 0u),
                                                   0, berr[i], est[i]};
        if (hinfo[i]) {  // singular low-precision factor: nothing to refine with
          full64.push_back(k[k0 + i]);
          full64_idx.push_back(r0 + (int64_t)i * ndir);
          full64_dir.push_back(d);
        } else if (!conv || sensitive) {
          flagged.push_back(i);
        }
      }
      // several directions: FP64 re-assembly (for this direction) and refinement with the existing
      // factor, in groups, batch by batch
      for (size_t f0 = 0; multi && f0 < flagged.size(); f0 += G) {
        const int ng = (int)std::min<size_t>(G, flagged.size() - f0);
        std::vector<double> kv(ng);
        for (int g = 0; g < ng; ++g) kv[g] = k[k0 + flagged[f0 + g]];
        BIE_CUDA_TRY(cudaMemcpyAsync(kg, kv.data(), ng * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        BIE_CUDA_TRY(cudaMemcpyAsync(sel_g, flagged.data() + f0, ng * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        BIE_TRY(mark(4));
        BIE_TRY(assemble64(c, kg, ng, A64, b64, s64, c->reassembly_ff != 0));
        BIE_TRY(refine_fp64_system(c, A64, b64, LU, ld, bstride, perm, sel_g, ng, (int)N, x, xg, rg, rowabs_g, state_g,
                                   c->refine64_it_max, c->refine64_tol, Dinv, s64, true));
        BIE_TRY(mark(5));
        BIE_TRY(refine_read_state(c, state_g, ng, gd.data(), gi.data(), gb.data(), ge.data()));
        if (timing) {
          c->phase.reassembly_ms += elapsed(4, 5);
          c->phase.reassembled += ng;
        }
        for (int g = 0; g < ng; ++g) {
          const int64_t idx = r0 + (int64_t)flagged[f0 + g] * ndir;
          if (rep) {
            rep[idx].flags |= BIE_FLAG_FP64_ASSEMBLY;
            rep[idx].iters += gi[g];
            rep[idx].backward_err = gb[g];
            if (gd[g]) rep[idx].flags &= ~BIE_FLAG_NOT_CONVERGED;
          }
          if (!gd[g] || !std::isfinite(gb[g])) {
            full64.push_back(k[k0 + flagged[f0 + g]]);
            full64_idx.push_back(idx);
            full64_dir.push_back(d);
          }
        }
      }
      dim3 g((unsigned)((N + 255) / 256), nk);
      BIE_LAUNCH(k_surface_fields<<<g, 256, 0, c->stream>>>(c->bc, N, x, known, surf_out + r0 * 2 * N, kstride));
      BIE_CUDA_TRY(cudaGetLastError());
      // (after the batch's surface values, which a flush of the pool overwrites for its systems)
      if (!multi) {  // into the pool (flushed when full and after the last batch)
        for (const int i : flagged) {
          if ((int)pool_k.size() == G) BIE_TRY(flush_pool());
          const int64_t slot = (int64_t)pool_k.size();
          BIE_CUDA_TRY(cudaMemcpyAsync(pLU + slot * bstride, LU + (int64_t)i * bstride, mat, cudaMemcpyDeviceToDevice,
                                       c->stream));
          BIE_CUDA_TRY(cudaMemcpyAsync(pperm + slot * N, perm + (int64_t)i * N, (size_t)N * 4, cudaMemcpyDeviceToDevice,
                                       c->stream));
          BIE_CUDA_TRY(cudaMemcpyAsync(pD + slot * dstride, Dinv + (int64_t)i * dstride, (size_t)dstride * sizeof(cf),
                                       cudaMemcpyDeviceToDevice, c->stream));
          BIE_CUDA_TRY(cudaMemcpyAsync(px + slot * N, x + (int64_t)i * N, (size_t)N * sizeof(cd),
                                       cudaMemcpyDeviceToDevice, c->stream));
          BIE_CUDA_TRY(cudaMemcpyAsync(pknown + slot * N, known + (int64_t)i * N, (size_t)N * sizeof(cd),
                                       cudaMemcpyDeviceToDevice, c->stream));
          pool_k.push_back(k[k0 + i]);
          pool_idx.push_back(r0 + (int64_t)i * ndir);
        }
      }
    }
    set_dir(0);
  }
  BIE_TRY(flush_pool());
  // Wavenumbers whose TF32 factor could not be refined against the FP64 re-assembly (cond(A)
  // times the TF32 factor's error near 1): the FP64 system is factored again in FP32 on the CUDA
  // cores (8000 times smaller factor error than TF32) and refined against itself with that factor;
  // only if that also stalls does the full FP64 path (an FP64 LU: about 70 times slower on this
  // GPU's FP64 pipe) solve it.  The batch buffers (slot 0) are free by now.
  std::vector<int32_t> one{0};
  for (size_t f = 0; c->refactor32 && f < full64.size(); ++f) {
    set_dir(full64_dir[f]);
    BIE_CUDA_TRY(cudaMemcpyAsync(kg, &full64[f], sizeof(double), cudaMemcpyHostToDevice, c->stream));
    BIE_CUDA_TRY(cudaMemcpyAsync(sel_g, one.data(), sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    BIE_TRY(assemble64(c, kg, 1, A64, b64, s64, c->reassembly_ff != 0));
    BIE_LAUNCH(k_cd_to_cf<<<dim3((unsigned)((N + 255) / 256), (unsigned)N), 256, 0, c->stream>>>(A64, N, LU, ld));
    BIE_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), c->stream));
    BIE_TRY(lu_factor32_panels(c, LU, 1, (int)N, (int)ld, bstride, piv, info, (char*)tcs + 256, (int32_t*)tcs));
    BIE_TRY(factor_aux(c, LU, 1, (int)N, ld, bstride, piv, perm, Dinv));
    BIE_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)N * sizeof(cd), c->stream));
    BIE_TRY(refine_fp64_system(c, A64, b64, LU, ld, bstride, perm, sel_g, 1, (int)N, x, xg, rg, rowabs_g, state_g,
                               kRefactorItMax, c->refine64_tol, Dinv, s64 + N, true));
    int32_t d1 = 0, it1 = 0, zp = 0, terr = 0;
    double b1 = 0.0, e1 = 0.0;
    BIE_TRY(refine_read_state(c, state_g, 1, &d1, &it1, &b1, &e1));
    BIE_CUDA_TRY(cudaMemcpy(&zp, info, sizeof(int32_t), cudaMemcpyDeviceToHost));
    BIE_TRY(lu_tc_error(c, tcs, &terr));
    if (terr) return fail(BIE_ERR_TIMEOUT, "LU: a bounded wait in a cooperative panel gave up");
    if (!d1 || zp || !std::isfinite(b1)) continue;  // stays for the full FP64 path
    dim3 gs((unsigned)((N + 255) / 256), 1);
    BIE_LAUNCH(k_surface_fields<<<gs, 256, 0, c->stream>>>(c->bc, N, x, s64, surf_out + full64_idx[f] * 2 * N, 2 * N));
    if (rep) {
      bie_report& rr = rep[full64_idx[f]];
      rr.flags = (rr.flags & ~BIE_FLAG_NOT_CONVERGED) | BIE_FLAG_FP32_REFACTOR | BIE_FLAG_FP64_ASSEMBLY;
      rr.iters += it1;
      rr.backward_err = b1;
    }
    full64[f] = -1.0;  // done
  }
  // last resort: the full FP64 path
  for (size_t f = 0; f < full64.size(); ++f) {
    if (full64[f] < 0.0) continue;
    bie_report r64;
    set_dir(full64_dir[f]);
    BIE_TRY(solve_fp64(c, &full64[f], 1, surf_out + full64_idx[f] * 2 * N, &r64));
    if (rep) {  // the direct FP64 solve replaces the stalled refinement's outcome
      bie_report& rr = rep[full64_idx[f]];
      rr.flags = (rr.flags & ~BIE_FLAG_NOT_CONVERGED) | BIE_FLAG_FALLBACK_FP64 | r64.flags;
      rr.path = BIE_MODE_FP64;
      rr.backward_err = r64.backward_err;
    }
  }
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

}  // namespace bie
