// capi.cu -- the C ABI of include/bie.h: argument checks, device buffers, and the order in which
// the kernels of the other translation units run.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>

#include "bie_common.cuh"

namespace bie {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
void uncount_launches(int64_t n) { g_launches.fetch_sub((uint64_t)n, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  return (e == cudaErrorMemoryAllocation) ? BIE_ERR_OOM : BIE_ERR_CUDA;
}

int dev_alloc(bie_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 1), c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(BIE_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  return BIE_OK;
}

int device_free(bie_ctx* c, size_t* free_b) {
  size_t total = 0;
  BIE_CUDA_TRY(cudaMemGetInfo(free_b, &total));
  if (c->mem_budget > 0) *free_b = std::min(*free_b, c->mem_budget);
  return BIE_OK;
}

void dev_free(bie_ctx* c, void* p) {
  if (p) cudaFreeAsync(p, c->stream);
}

int ensure_buf(bie_ctx* c, DeviceBuf& b, size_t bytes) {
  if (b.bytes >= bytes) return BIE_OK;
  dev_free(c, b.p);
  b.p = nullptr;
  b.bytes = 0;
  BIE_TRY(dev_alloc(c, &b.p, bytes));
  b.bytes = bytes;
  return BIE_OK;
}
int smem_optin() {
  static std::atomic<int> v{0};
  int x = v.load();
  if (x == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&x, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || x <= 0)
      x = 48 * 1024;
    v.store(x);
  }
  return x;
}

int capture_begin(bie_ctx* c, cudaStream_t* saved) {
  if (!c->cap_stream) BIE_CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  BIE_CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed));
  *saved = c->stream;
  c->stream = c->cap_stream;
  return BIE_OK;
}

int capture_end(bie_ctx* c, cudaStream_t saved, cudaGraph_t* graph) {
  c->stream = saved;
  *graph = nullptr;
  BIE_CUDA_TRY(cudaStreamEndCapture(c->cap_stream, graph));
  return BIE_OK;
}

int ensure_pinned(bie_ctx* c, size_t bytes) {
  if (c->pinned_bytes >= bytes) return BIE_OK;
  if (c->pinned) {
    cudaStreamSynchronize(c->stream);
    cudaFreeHost(c->pinned);
    c->pinned = nullptr;
    c->pinned_bytes = 0;
  }
  BIE_CUDA_TRY(cudaMallocHost(&c->pinned, bytes));
  c->pinned_bytes = bytes;
  return BIE_OK;
}

void free_buf(bie_ctx* c, DeviceBuf& b) {
  dev_free(c, b.p);
  b.p = nullptr;
  b.bytes = 0;
}

// translation-unit entry points
int upload_geometry_tables(bie_ctx* c);
int build_colouring(bie_ctx* c);
int host_geometry_checks(bie_ctx* c, bool make_normals);
void build_quad_rule(QuadRule& r, int ng, int ng_near);
int launch_foot_points(bie_ctx* c, const double* xp, int64_t M, int32_t* foot_elem, double* foot,
                       unsigned long long* first_inside);
int assemble64(bie_ctx* c, const double* kv, int nk, cd* A, cd* b, void* scratch, bool ff_bulk);
int lu_factor64(bie_ctx* c, cd* A, int batch, int n, int ld, int64_t bstride, int32_t* piv, int32_t* info);
int lu_solve64(bie_ctx* c, const cd* LU, int batch, int n, int ld, int64_t bstride, const int32_t* piv, cd* b,
               int64_t bstride_b);
int field64(bie_ctx* c, const double* kv, int nk, const cd* surf, const double* xp, int64_t M,
            const int32_t* foot_elem, const double* foot, cd* T, void* scratch);
int pulse_spectrum(bie_ctx* c, const double* s, int64_t P, int n, cd* Sout);
int synthesize(bie_ctx* c, const cd* T, const int64_t* midx_dev, int nk, int64_t M, const cd* Sp, int64_t P, int n,
               void* out, int out_dtype);
int top_frequencies(bie_ctx* c, const cd* S, int64_t P, int nm, int K, int64_t* midx_dev);
int solve_fp64_linear(bie_ctx* c, const double* k, int64_t Nk, cd* surf_out, bie_report* rep);
int assemble_linear_one(bie_ctx* c, double k, cd* A_out, cd* b_out);
int expand_linear(bie_ctx* c, const cd* surf_lin, int nk, cd* surf_q);
int solve_mixed_async(bie_ctx* c, const double* k, int64_t Nk, cd* surf_out, bie_report* rep);
int solve_mixed(bie_ctx* c, const double* k, int64_t Nk, cd* surf_out, bie_report* rep, cf* lu_keep,
                int32_t* perm_keep, cf* d_keep, const double* dirs, int ndir);
int solve_learned(bie_ctx* c, const double* k, int64_t Nk, cd* surf_out, bie_report* rep);
void mlp_free(bie_ctx* c);
int mlp_set_params(bie_ctx* c, const float* theta_host);
int mlp_get_params(bie_ctx* c, float* theta_host);
int mlp_features_api(bie_ctx* c, const double* k, int64_t nk, float* phi);
int mlp_forward_api(bie_ctx* c, const float* X, int64_t B, float* Y);
int mlp_loss_grad_api(bie_ctx* c, const float* X, const float* T, int64_t B, float* grad, float* loss);
int mlp_adam_api(bie_ctx* c, const float* grad, double lr);
int mlp_train(bie_ctx* c, const double* k, int64_t nk, const cd* surf, int epochs, float* loss_hist);
int mlp_predict_api(bie_ctx* c, const double* k, int64_t nk, cd* x0);
int autotune(bie_ctx* c, const double* k, int64_t nk, const char* cache_path, bie_tune_result* out);
int field_mixed(bie_ctx* c, const double* kv, int nk, const cd* surf, const double* xp, int64_t M,
                const int32_t* foot_elem, const double* foot, cd* T, void* scratch, size_t scratch_bytes);

static void free_geometry(bie_ctx* c) {
  void* ptrs[] = {c->nodes, c->elems, c->normals, c->bc, c->qgeo, c->ngeo, c->qshape, c->nshape, c->qgeo32,
                  c->qshape32, c->nshape32, c->color_off, c->elem_perm, c->n2e_off, c->n2e, c->d_nnear, c->bc_flip,
                  c->lin_adj_off, c->lin_adj, c->lin_mid, c->win_lo, c->wcol_off};
  for (void* p : ptrs) dev_free(c, p);
  c->nodes = nullptr; c->elems = nullptr; c->normals = nullptr; c->bc = nullptr;
  c->qgeo = nullptr; c->ngeo = nullptr; c->qshape = nullptr; c->nshape = nullptr;
  c->qgeo32 = nullptr; c->qshape32 = nullptr; c->nshape32 = nullptr; c->color_off = nullptr; c->elem_perm = nullptr;
  c->n2e_off = nullptr; c->n2e = nullptr; c->d_nnear = nullptr; c->bc_flip = nullptr;
  c->lin_adj_off = nullptr; c->lin_adj = nullptr; c->lin_mid = nullptr; c->lin_N = 0;
  c->win_lo = nullptr; c->wcol_off = nullptr; c->nwin = 0; c->win_max = 0;
  c->far_r2 = 0.0;
  c->uniform_bc = -1;
  c->has_geom = false;
}

// P, P' at every node from the solution vector and the known boundary values.
// surf: [nk] blocks of [2][N], kstride elements apart (2N, or 2N x directions).
__global__ void k_surface_fields(const uint8_t* __restrict__ bc, int64_t N, const cd* __restrict__ x,
                                 const cd* __restrict__ known, cd* __restrict__ surf, int64_t kstride) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int kk = blockIdx.y;
  if (j >= N) return;
  cd xv = x[(int64_t)kk * N + j], kv = known[(int64_t)kk * N + j];
  cd* s = surf + (int64_t)kk * kstride;
  if (bc[j] == 0) { s[j] = xv; s[N + j] = kv; }
  else { s[j] = kv; s[N + j] = xv; }
}

static int check_ctx(bie_ctx* c, bool need_geom) {
  if (!c) return fail(BIE_ERR_INVALID_ARG, "NULL context");
  if (need_geom && !c->has_geom) return fail(BIE_ERR_STATE, "no geometry: call bie_set_geometry first");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return BIE_OK;
}

// k = 0 is the zero-frequency term of Eq. (inverseFourier), solved by the k -> 0 limit of the same
// kernels (f -> nu.r); positive k below 1e-30 would overflow 1/k in FP32 and are rejected.
static int check_k(const double* k, int64_t Nk, bool allow_zero = true) {
  if (Nk < 0) return fail(BIE_ERR_INVALID_ARG, "Nk < 0");
  if (Nk > 0 && !k) return fail(BIE_ERR_INVALID_ARG, "NULL k");
  for (int64_t i = 0; i < Nk; ++i) {
    if (!std::isfinite(k[i]) || k[i] < 0.0 || (k[i] > 0.0 && k[i] < 1e-30) || (!allow_zero && k[i] == 0.0))
      return fail(BIE_ERR_INVALID_ARG, "k[" + std::to_string(i) + "] must be finite and " +
                                           (allow_zero ? "either 0 or >= 1e-30" : ">= 1e-30"));
  }
  return BIE_OK;
}

// The boundary conditions exchanged at every node (device, made once per geometry): assembling
// with them gives the known-column matrix of the real conditions.
int flipped_bc(bie_ctx* c, uint8_t** out) {
  if (!c->bc_flip) {
    std::vector<uint8_t> f(c->N);
    for (int64_t j = 0; j < c->N; ++j) f[j] = (uint8_t)(1 - c->h_bc[j]);
    BIE_TRY(dev_alloc(c, (void**)&c->bc_flip, c->N));
    BIE_CUDA_TRY(cudaMemcpyAsync(c->bc_flip, f.data(), c->N, cudaMemcpyHostToDevice, c->stream));
  }
  *out = c->bc_flip;
  return BIE_OK;
}

int rhs_from_known64(bie_ctx* c, const cd* B, int nk, int n, const cd* known, cd* zero, cd* b, double* rowabs,
                     void* state_dev);
size_t refine_state_bytes(int nk);
__global__ void k_known64(const double* __restrict__ nodes, const double* __restrict__ normals,
                          const uint8_t* __restrict__ bc, int64_t N, const double* __restrict__ kv, double dx,
                          double dy, double dz, cd* __restrict__ known);

// Several incident directions in FP64 (see solve_mixed): A and the known-column matrix B assembled
// once per wavenumber, A factored once, b_d = -B known_d per direction.  surf_out [Nk][ndir][2][N].
int solve_fp64_multi(bie_ctx* c, const double* k, int64_t Nk, const double* dirs, int ndir, cd* surf_out,
                     bie_report* rep) {
  const int64_t N = c->N;
  uint8_t* bc_flip = nullptr;
  BIE_TRY(flipped_bc(c, &bc_flip));
  const double dir0[3] = {c->dir[0], c->dir[1], c->dir[2]};
  struct DirGuard {
    bie_ctx* c;
    double d[3];
    ~DirGuard() { for (int t = 0; t < 3; ++t) c->dir[t] = d[t]; }
  } dirguard{c, {dir0[0], dir0[1], dir0[2]}};
  auto set_dir = [&](int d) { for (int t = 0; t < 3; ++t) c->dir[t] = dirs[3 * d + t]; };
  const size_t st_bytes = (refine_state_bytes(1) + 15) / 16 * 16;
  const size_t perk = 2 * (size_t)N * N * sizeof(cd) + (size_t)N * sizeof(cd) * 8 + (size_t)N * sizeof(double) +
                      (size_t)N * 4 + st_bytes + 64;
  size_t free_b = 0;
  BIE_TRY(device_free(c, &free_b));
  int64_t kb = std::max<int64_t>(1, std::min<int64_t>(Nk, std::min<int64_t>(256, (int64_t)((free_b / 2) / perk))));
  if ((size_t)kb * perk > free_b) return fail(BIE_ERR_OOM, "two FP64 matrices of N = " + std::to_string(N) + " do not fit");
  BIE_TRY(ensure_buf(c, c->work, kb * perk + 4096));
  char* base = (char*)c->work.p;
  cd* A = (cd*)base;
  cd* Bm = A + kb * N * N;
  cd* b = Bm + kb * N * N;
  cd* scratch = b + kb * N;  // known [kb][N], rowsum [kb][N][3]
  cd* bd = scratch + kb * N * 4;
  cd* zero = bd + kb * N;
  cd* known = zero + kb * N;
  double* rowabs = (double*)(known + kb * N);
  int32_t* piv = (int32_t*)(rowabs + kb * N);
  int32_t* info = piv + kb * N;
  char* stp = (char*)(((uintptr_t)(info + kb) + 15) & ~(uintptr_t)15);
  void* state = stp;
  double* kdev = (double*)(stp + kb * st_bytes);
  std::vector<int32_t> hinfo(kb);
  for (int64_t k0 = 0; k0 < Nk; k0 += kb) {
    const int nk = (int)std::min<int64_t>(kb, Nk - k0);
    BIE_CUDA_TRY(cudaMemcpyAsync(kdev, k + k0, nk * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    BIE_CUDA_TRY(cudaMemsetAsync(info, 0, nk * sizeof(int32_t), c->stream));
    set_dir(0);
    uint8_t* bc_real = c->bc;
    c->bc = bc_flip;
    int rc = assemble64(c, kdev, nk, Bm, bd, scratch, false);  // b and known of this call: discarded
    c->bc = bc_real;
    BIE_TRY(rc);
    BIE_TRY(assemble64(c, kdev, nk, A, b, scratch, false));
    BIE_TRY(lu_factor64(c, A, nk, (int)N, (int)N, N * N, piv, info));
    for (int d = 0; d < ndir; ++d) {
      set_dir(d);
      dim3 gk((unsigned)((N + 255) / 256), nk);
      BIE_LAUNCH(k_known64<<<gk, 256, 0, c->stream>>>(c->nodes, c->normals, c->bc, N, kdev, c->dir[0], c->dir[1],
                                                     c->dir[2], known));
      BIE_TRY(rhs_from_known64(c, Bm, nk, (int)N, known, zero, bd, rowabs, state));
      BIE_TRY(lu_solve64(c, A, nk, (int)N, (int)N, N * N, piv, bd, N));
      dim3 g((unsigned)((N + 255) / 256), nk);
      BIE_LAUNCH(k_surface_fields<<<g, 256, 0, c->stream>>>(c->bc, N, bd, known, surf_out + (k0 * ndir + d) * 2 * N,
                                                           (int64_t)ndir * 2 * N));
      BIE_CUDA_TRY(cudaGetLastError());
    }
    if (rep) {
      BIE_CUDA_TRY(cudaMemcpyAsync(hinfo.data(), info, nk * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
      BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
      for (int i = 0; i < nk; ++i)
        for (int d = 0; d < ndir; ++d)
          rep[(k0 + i) * ndir + d] = bie_report{0, BIE_MODE_FP64, hinfo[i] ? BIE_FLAG_ZERO_PIVOT : 0u, 0, 0.0, 0.0};
    }
  }
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

int solve_fp64(bie_ctx* c, const double* k, int64_t Nk, cd* surf_out, bie_report* rep) {
  const int64_t N = c->N;
  const size_t perk = (size_t)N * N * sizeof(cd) + (size_t)N * sizeof(cd) * 6 + (size_t)N * 4 + 64;
  size_t free_b = 0;
  BIE_TRY(device_free(c, &free_b));
  int64_t kb = std::max<int64_t>(1, std::min<int64_t>(Nk, std::min<int64_t>(256, (int64_t)((free_b / 2) / perk))));
  if ((size_t)kb * perk > free_b) return fail(BIE_ERR_OOM, "one FP64 system of N = " + std::to_string(N) + " does not fit in device memory");
  BIE_TRY(ensure_buf(c, c->work, kb * perk + 4096));
  char* base = (char*)c->work.p;
  cd* A = (cd*)base;
  cd* b = A + kb * N * N;
  cd* scratch = b + kb * N;  // known [kb][N], rowsum [kb][N][3]
  int32_t* piv = (int32_t*)(scratch + kb * N * 4);
  int32_t* info = piv + kb * N;
  double* kdev = (double*)(((uintptr_t)(info + kb) + 15) & ~(uintptr_t)15);
  std::vector<int32_t> hinfo(kb);
  for (int64_t k0 = 0; k0 < Nk; k0 += kb) {
    const int nk = (int)std::min<int64_t>(kb, Nk - k0);
    BIE_CUDA_TRY(cudaMemcpyAsync(kdev, k + k0, nk * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    BIE_CUDA_TRY(cudaMemsetAsync(info, 0, nk * sizeof(int32_t), c->stream));
    BIE_TRY(assemble64(c, kdev, nk, A, b, scratch, false));
    BIE_TRY(lu_factor64(c, A, nk, (int)N, (int)N, N * N, piv, info));
    BIE_TRY(lu_solve64(c, A, nk, (int)N, (int)N, N * N, piv, b, N));
    dim3 g((unsigned)((N + 255) / 256), nk);
    BIE_LAUNCH(k_surface_fields<<<g, 256, 0, c->stream>>>(c->bc, N, b, scratch, surf_out + k0 * 2 * N, 2 * N));
    BIE_CUDA_TRY(cudaGetLastError());
    if (rep) {
      BIE_CUDA_TRY(cudaMemcpyAsync(hinfo.data(), info, nk * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
      BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
      for (int i = 0; i < nk; ++i) {
        rep[k0 + i] = bie_report{0, BIE_MODE_FP64, hinfo[i] ? BIE_FLAG_ZERO_PIVOT : 0u, 0, 0.0, 0.0};
      }
    }
  }
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

}  // namespace bie

using namespace bie;

extern "C" {

const char* bie_last_error(void) { return g_last_error.c_str(); }

const char* bie_version(void) { return "bie-gb300 0.1 (sm_103a)"; }

uint64_t bie_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int bie_create(bie_ctx** out, int cuda_device, void* cuda_stream) {
  if (!out) return fail(BIE_ERR_INVALID_ARG, "NULL out");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (cuda_device < 0 || cuda_device >= n)
    return fail(BIE_ERR_INVALID_ARG, "device " + std::to_string(cuda_device) + " out of range (" + std::to_string(n) + " devices)");
  e = cudaSetDevice(cuda_device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  bie_ctx* c = new (std::nothrow) bie_ctx();
  if (!c) return fail(BIE_ERR_OOM, "host allocation failed");
  c->device = cuda_device;
  c->stream = (cudaStream_t)cuda_stream;
  *out = c;
  return BIE_OK;
}

int bie_destroy(bie_ctx* c) {
  if (!c) return BIE_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  free_geometry(c);
  free_buf(c, c->work);
  free_buf(c, c->work2);
  free_buf(c, c->work3);
  free_buf(c, c->work4);
  free_buf(c, c->work5);
  free_buf(c, c->work6);
  mlp_free(c);
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->rep_pinned) cudaFreeHost(c->rep_pinned);
  for (void* q : c->rep_pinned_old) cudaFreeHost(q);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
  return BIE_OK;
}

int bie_set_quadrature(bie_ctx* c, int ng, int ng_near) {
  BIE_TRY(check_ctx(c, false));
  if (ng < 1 || ng > 8 || ng_near < 1 || ng_near > 12)
    return fail(BIE_ERR_INVALID_ARG, "quadrature orders must satisfy 1 <= ng <= 8, 1 <= ng_near <= 12");
  c->ng = ng;
  c->ng_near = ng_near;
  return BIE_OK;
}

int bie_set_option(bie_ctx* c, const char* name, double value) {
  BIE_TRY(check_ctx(c, false));
  if (!name) return fail(BIE_ERR_INVALID_ARG, "NULL option name");
  const std::string n(name);
  if (!std::isfinite(value)) return fail(BIE_ERR_INVALID_ARG, "option value must be finite");
  if (n == "mixed.tcgen05") {
    if (value != 0.0 && value != 1.0 && value != 2.0 && value != 3.0)
      return fail(BIE_ERR_INVALID_ARG, "mixed.tcgen05 must be 0 (SIMT), 1, 2 or 3 (tensor-core kernels)");
    c->tc_version = (int)value;
  } else if (n == "mixed.lu_block") {
    if (value != 0.0 && value != 128.0 && value != 256.0 && value != 512.0)
      return fail(BIE_ERR_INVALID_ARG, "mixed.lu_block must be 0 (by N), 128, 256 or 512");
    c->lu_block = (int)value;
  } else if (n == "asm.windows") {
    c->asm_windows = value != 0.0 ? 1 : 0;
  } else if (n == "mixed.reassembly_group") {
    if (value < 1 || value > 32) return fail(BIE_ERR_INVALID_ARG, "mixed.reassembly_group must be in [1, 32]");
    c->reassembly_group = (int)value;
  } else if (n == "mixed.lu_coop") {
    c->lu_coop = value != 0.0 ? 1 : 0;
  } else if (n == "mixed.lu_tile") {
    if (value != 128.0 && value != 256.0) return fail(BIE_ERR_INVALID_ARG, "mixed.lu_tile must be 128 or 256");
    c->lu_tile = (int)value;
  } else if (n == "mixed.lu_panel") {
    if (value != 32.0 && value != 64.0) return fail(BIE_ERR_INVALID_ARG, "mixed.lu_panel must be 32 or 64");
    c->lu_panel = (int)value;
  } else if (n == "mixed.batch") {
    if (value < 1 || value > 4096) return fail(BIE_ERR_INVALID_ARG, "mixed.batch must be in [1, 4096]");
    c->mixed_batch = (int)value;
  } else if (n == "refine.tol") {
    if (!(value > 0.0) || value >= 1.0) return fail(BIE_ERR_INVALID_ARG, "refine.tol must be in (0, 1)");
    c->refine_tol = value;
  } else if (n == "refine.it_max") {
    if (value < 0 || value > 64) return fail(BIE_ERR_INVALID_ARG, "refine.it_max must be in [0, 64]");
    c->refine_it_max = (int)value;
  } else if (n == "mixed.refactor32") {
    c->refactor32 = value != 0.0 ? 1 : 0;
  } else if (n == "mixed.refine64_it_max") {
    if (value < 0 || value > 64) return fail(BIE_ERR_INVALID_ARG, "mixed.refine64_it_max must be in [0, 64]");
    c->refine64_it_max = (int)value;
  } else if (n == "mixed.fallback_err_est") {
    if (!(value > 0.0)) return fail(BIE_ERR_INVALID_ARG, "mixed.fallback_err_est must be > 0");
    c->fallback_err_est = value;
  } else if (n == "field.accurate_phase") {
    c->field_accurate_phase = value != 0.0 ? 1 : 0;
  } else if (n == "field.variant") {
    if (value != 0.0 && value != 1.0 && value != 2.0)
      return fail(BIE_ERR_INVALID_ARG, "field.variant must be 0, 1 or 2");
    c->field_variant = (int)value;
  } else if (n == "mixed.asm_kb") {
    if (value != 0.0 && value != 1.0 && value != 2.0) return fail(BIE_ERR_INVALID_ARG, "mixed.asm_kb must be 0, 1 or 2");
    c->asm_kb = (int)value;
  } else if (n == "assemble.bulk_ff") {
    c->assemble_ff = value != 0.0 ? 1 : 0;
  } else if (n == "mixed.reassembly") {
    if (value != 0.0 && value != 1.0) return fail(BIE_ERR_INVALID_ARG, "mixed.reassembly must be 0 (FP64) or 1 (float-float)");
    c->reassembly_ff = (int)value;
  } else if (n == "mixed.graph") {
    c->mixed_graph = value != 0.0 ? 1 : 0;
  } else if (n == "mixed.phase_timing") {
    c->phase_timing = value != 0.0 ? 1 : 0;
  } else if (n == "learned.stride") {
    if (value < 2 || value > 1e6) return fail(BIE_ERR_INVALID_ARG, "learned.stride must be in [2, 1e6]");
    c->learned_stride = (int)value;
  } else if (n == "learned.x0") {
    if (value != 0.0 && value != 1.0 && value != 2.0 && value != 3.0)
      return fail(BIE_ERR_INVALID_ARG,
                  "learned.x0 must be 0 (zero), 1 (network), 2 (nearest anchor) or 3 (anchor interpolant)");
    c->learned_x0 = (int)value;
  } else if (n == "learned.epochs") {
    if (value < 0 || value > 100000) return fail(BIE_ERR_INVALID_ARG, "learned.epochs must be in [0, 100000]");
    c->mlp_epochs = (int)value;
  } else if (n == "learned.batch") {
    if (value < 128 || value > 1048576) return fail(BIE_ERR_INVALID_ARG, "learned.batch must be in [128, 1048576]");
    c->mlp_batch = (int)((((int64_t)value) + 127) / 128 * 128);
  } else if (n == "learned.lr") {
    if (!(value > 0.0) || value > 1.0) return fail(BIE_ERR_INVALID_ARG, "learned.lr must be in (0, 1]");
    c->mlp_lr = value;
  } else if (n == "learned.lr_min") {
    if (!(value >= 0.0) || value > 1.0) return fail(BIE_ERR_INVALID_ARG, "learned.lr_min must be in [0, 1]");
    c->mlp_lr_min = value;
  } else if (n == "learned.seed") {
    if (value < 0 || value > 9.0e15) return fail(BIE_ERR_INVALID_ARG, "learned.seed must be in [0, 9e15]");
    c->mlp_seed = (int64_t)value;
  } else if (n == "learned.kmax") {
    if (value < 0) return fail(BIE_ERR_INVALID_ARG, "learned.kmax must be >= 0");
    c->mlp_kmax = value;
  } else if (n == "learned.graph") {
    c->mlp_graph = value != 0.0 ? 1 : 0;
  } else if (n == "gmres.m") {
    if (value < 1 || value > 62) return fail(BIE_ERR_INVALID_ARG, "gmres.m must be in [1, 62]");
    c->gmres_m = (int)value;
  } else if (n == "gmres.cycles") {
    if (value < 1 || value > 100) return fail(BIE_ERR_INVALID_ARG, "gmres.cycles must be in [1, 100]");
    c->gmres_cycles = (int)value;
  } else if (n == "gmres.inner_tol") {
    if (!(value > 0.0) || value >= 1.0) return fail(BIE_ERR_INVALID_ARG, "gmres.inner_tol must be in (0, 1)");
    c->gmres_inner_tol = value;
  } else {
    return fail(BIE_ERR_INVALID_ARG, "unknown option '" + n + "'");
  }
  return BIE_OK;
}

int bie_set_incident_plane_wave(bie_ctx* c, const double* dir) {
  BIE_TRY(check_ctx(c, false));
  if (!dir) return fail(BIE_ERR_INVALID_ARG, "NULL direction");
  double n = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  if (!(n > 0.0) || !std::isfinite(n)) return fail(BIE_ERR_INVALID_ARG, "direction must be finite and non-zero");
  for (int d = 0; d < 3; ++d) c->dir[d] = dir[d] / n;
  return BIE_OK;
}

int set_geometry_impl(bie_ctx* c, const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                      const double* normals, const uint8_t* bc) {
  if (!nodes || !elems || !bc) return fail(BIE_ERR_INVALID_ARG, "NULL nodes, elems or bc");
  if (N < 3 || E < 1) return fail(BIE_ERR_INVALID_ARG, "need N >= 3 and E >= 1");
  if (N > (int64_t)1 << 30 || E > (int64_t)1 << 28) return fail(BIE_ERR_INVALID_ARG, "mesh too large");
  cudaStreamSynchronize(c->stream);
  free_geometry(c);
  c->N = N;
  c->E = E;
  c->h_nodes.assign(nodes, nodes + 3 * N);
  c->h_elems.assign(elems, elems + 6 * E);
  c->h_bc.assign(bc, bc + N);
  for (int64_t i = 0; i < N; ++i)
    if (c->h_bc[i] > 1) return fail(BIE_ERR_INVALID_ARG, "bc values must be 0 (hard) or 1 (soft)");
  if (normals) c->h_normals.assign(normals, normals + 3 * N);
  BIE_TRY(host_geometry_checks(c, normals == nullptr));
  build_quad_rule(c->rule, c->ng, c->ng_near);
  BIE_TRY(dev_alloc(c, (void**)&c->nodes, 3 * N * sizeof(double)));
  BIE_TRY(dev_alloc(c, (void**)&c->normals, 3 * N * sizeof(double)));
  BIE_TRY(dev_alloc(c, (void**)&c->elems, 6 * E * sizeof(int32_t)));
  BIE_TRY(dev_alloc(c, (void**)&c->bc, N));
  BIE_TRY(dev_alloc(c, (void**)&c->d_nnear, 6 * sizeof(int)));
  // the host copies live in the context, so the asynchronous uploads may outlive this call
  BIE_CUDA_TRY(cudaMemcpyAsync(c->nodes, c->h_nodes.data(), 3 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaMemcpyAsync(c->normals, c->h_normals.data(), 3 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaMemcpyAsync(c->elems, c->h_elems.data(), 6 * E * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaMemcpyAsync(c->bc, c->h_bc.data(), N, cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaMemcpyAsync(c->d_nnear, c->rule.nnear, 6 * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  BIE_TRY(build_colouring(c));
  BIE_TRY(upload_geometry_tables(c));
  c->has_geom = true;
  return BIE_OK;
}

int bie_set_geometry(bie_ctx* c, const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                     const double* normals, const uint8_t* bc) {
  BIE_TRY(check_ctx(c, false));
  return set_geometry_impl(c, nodes, N, elems, E, normals, bc);
}

int bie_assemble(bie_ctx* c, double k, void* A_out, void* b_out) {
  BIE_TRY(check_ctx(c, true));
  if (!A_out || !b_out) return fail(BIE_ERR_INVALID_ARG, "NULL output");
  BIE_TRY(check_k(&k, 1));
  if (c->lin_N > 0) return assemble_linear_one(c, k, (cd*)A_out, (cd*)b_out);
  const int64_t N = c->N;
  BIE_TRY(ensure_buf(c, c->work, (size_t)N * 4 * sizeof(cd) + 64));
  double* kdev = (double*)((char*)c->work.p + (size_t)N * 4 * sizeof(cd));
  BIE_CUDA_TRY(cudaMemcpyAsync(kdev, &k, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  BIE_TRY(assemble64(c, kdev, 1, (cd*)A_out, (cd*)b_out, c->work.p, c->assemble_ff != 0));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

int bie_solve_frequencies(bie_ctx* c, const double* k, int64_t Nk, int mode, void* surf_out, bie_report* rep) {
  BIE_TRY(check_ctx(c, true));
  BIE_TRY(check_k(k, Nk, mode != BIE_MODE_LEARNED));
  if (Nk == 0) return BIE_OK;
  if (!surf_out) return fail(BIE_ERR_INVALID_ARG, "NULL surf_out");
  if (c->lin_N > 0) {
    if (mode != BIE_MODE_FP64) return fail(BIE_ERR_INVALID_ARG, "linear elements: BIE_MODE_FP64 only");
    return solve_fp64_linear(c, k, Nk, (cd*)surf_out, rep);
  }
  if (mode == BIE_MODE_FP64) return solve_fp64(c, k, Nk, (cd*)surf_out, rep);
  if (mode == BIE_MODE_MIXED) return solve_mixed(c, k, Nk, (cd*)surf_out, rep, nullptr, nullptr, nullptr, nullptr, 1);
  if (mode == BIE_MODE_LEARNED) return solve_learned(c, k, Nk, (cd*)surf_out, rep);
  return fail(BIE_ERR_INVALID_ARG, "unknown mode " + std::to_string(mode));
}

int bie_solve_frequencies_async(bie_ctx* c, const double* k, int64_t Nk, int mode, void* surf_out, bie_report* rep) {
  BIE_TRY(check_ctx(c, true));
  BIE_TRY(check_k(k, Nk, true));
  if (Nk == 0) return BIE_OK;
  if (!surf_out) return fail(BIE_ERR_INVALID_ARG, "NULL surf_out");
  if (c->lin_N > 0) return fail(BIE_ERR_INVALID_ARG, "linear elements: bie_solve_frequencies (BIE_MODE_FP64) only");
  if (mode != BIE_MODE_MIXED) return fail(BIE_ERR_INVALID_ARG, "bie_solve_frequencies_async: BIE_MODE_MIXED only");
  return solve_mixed_async(c, k, Nk, (cd*)surf_out, rep);
}

// ---- learned warm start ----------------------------------------------------------------------
int bie_mlp_set_params(bie_ctx* c, const float* theta) {
  BIE_TRY(check_ctx(c, false));
  if (!theta) return fail(BIE_ERR_INVALID_ARG, "NULL theta");
  for (int64_t i = 0; i < BIE_MLP_PARAMS; ++i)
    if (!std::isfinite(theta[i])) return fail(BIE_ERR_INVALID_ARG, "non-finite parameter at " + std::to_string(i));
  return mlp_set_params(c, theta);
}

int bie_mlp_get_params(bie_ctx* c, float* theta) {
  BIE_TRY(check_ctx(c, false));
  if (!theta) return fail(BIE_ERR_INVALID_ARG, "NULL theta");
  return mlp_get_params(c, theta);
}

int bie_mlp_features(bie_ctx* c, const double* k, int64_t nk, float* phi_out) {
  BIE_TRY(check_ctx(c, true));
  BIE_TRY(check_k(k, nk));
  if (nk > 0 && !phi_out) return fail(BIE_ERR_INVALID_ARG, "NULL phi_out");
  return mlp_features_api(c, k, nk, phi_out);
}

int bie_mlp_forward(bie_ctx* c, const float* X, int64_t B, float* Y_out) {
  BIE_TRY(check_ctx(c, false));
  if (B < 0 || B > ((int64_t)1 << 26)) return fail(BIE_ERR_INVALID_ARG, "B out of range");
  if (B > 0 && (!X || !Y_out)) return fail(BIE_ERR_INVALID_ARG, "NULL pointer");
  return mlp_forward_api(c, X, B, Y_out);
}

int bie_mlp_loss_grad(bie_ctx* c, const float* X, const float* T, int64_t B, float* grad_out, float* loss_out) {
  BIE_TRY(check_ctx(c, false));
  if (B < 1 || B > ((int64_t)1 << 26)) return fail(BIE_ERR_INVALID_ARG, "B out of range");
  if (!X || !T) return fail(BIE_ERR_INVALID_ARG, "NULL pointer");
  return mlp_loss_grad_api(c, X, T, B, grad_out, loss_out);
}

int bie_mlp_adam_step(bie_ctx* c, const float* grad, double lr) {
  BIE_TRY(check_ctx(c, false));
  if (!grad) return fail(BIE_ERR_INVALID_ARG, "NULL grad");
  if (!(lr > 0.0) || !std::isfinite(lr)) return fail(BIE_ERR_INVALID_ARG, "lr must be finite and > 0");
  return mlp_adam_api(c, grad, lr);
}

int bie_mlp_train(bie_ctx* c, const double* k, int64_t nk, const void* surf, int epochs, float* loss_hist) {
  BIE_TRY(check_ctx(c, true));
  BIE_TRY(check_k(k, nk));
  if (nk < 1 || !surf) return fail(BIE_ERR_INVALID_ARG, "need nk >= 1 and surf");
  if (epochs < 0 || epochs > 100000) return fail(BIE_ERR_INVALID_ARG, "epochs out of range");
  BIE_TRY(mlp_train(c, k, nk, (const cd*)surf, epochs, loss_hist));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

int bie_mlp_predict(bie_ctx* c, const double* k, int64_t nk, void* x0_out) {
  BIE_TRY(check_ctx(c, true));
  BIE_TRY(check_k(k, nk));
  if (nk > 0 && !x0_out) return fail(BIE_ERR_INVALID_ARG, "NULL x0_out");
  return mlp_predict_api(c, k, nk, (cd*)x0_out);
}

int bie_autotune(bie_ctx* c, const double* k, int64_t nk, const char* cache_path, bie_tune_result* out) {
  BIE_TRY(check_ctx(c, true));
  BIE_TRY(check_k(k, nk));
  return autotune(c, k, nk, cache_path, out);
}

int bie_get_phase_times(bie_ctx* c, bie_phase_times* out) {
  BIE_TRY(check_ctx(c, false));
  if (!out) return fail(BIE_ERR_INVALID_ARG, "NULL out");
  *out = c->phase;
  return BIE_OK;
}

int bie_get_learned_info(bie_ctx* c, bie_learned_info* out) {
  BIE_TRY(check_ctx(c, false));
  if (!out) return fail(BIE_ERR_INVALID_ARG, "NULL out");
  *out = c->learned_info;
  return BIE_OK;
}

int bie_eval_field(bie_ctx* c, const double* xobs, int64_t M, const double* k, int64_t Nk, const void* surf,
                   int mode, void* T_out) {
  BIE_TRY(check_ctx(c, true));
  BIE_TRY(check_k(k, Nk));
  if (M < 0) return fail(BIE_ERR_INVALID_ARG, "M < 0");
  if (M == 0 || Nk == 0) return BIE_OK;
  if (!xobs || !surf || !T_out) return fail(BIE_ERR_INVALID_ARG, "NULL pointer");
  if (mode != BIE_MODE_FP64 && mode != BIE_MODE_MIXED) return fail(BIE_ERR_INVALID_ARG, "unknown mode");
  const int64_t EQ = c->E * c->rule.Q;
  // foot points (k independent) then batches of k
  const size_t foot_bytes = (size_t)M * (8 * sizeof(double) + sizeof(int32_t)) + 256;
  const size_t perk = 2 * (size_t)EQ * sizeof(cd) + 16;
  // up to 512 wavenumbers per launch: the field kernel's grid (points x groups of 16 wavenumbers)
  // then spans many waves of resident CTAs, so the last, partial wave costs little
  constexpr int64_t kMaxFieldBatch = 512;
  int64_t kb = std::max<int64_t>(1, std::min<int64_t>(Nk, kMaxFieldBatch));
  BIE_TRY(ensure_buf(c, c->work3, foot_bytes + kb * perk + kMaxFieldBatch * sizeof(double) + 4096 + 256));
  double* foot = (double*)c->work3.p;
  int32_t* foot_elem = (int32_t*)(foot + 8 * M);
  char* after = (char*)(((uintptr_t)(foot_elem + M) + 255) & ~(uintptr_t)255);
  unsigned long long* first_inside = (unsigned long long*)after;
  after += 256;
  double* kdev = (double*)after;
  void* scratch = (void*)(after + kMaxFieldBatch * sizeof(double));
  BIE_CUDA_TRY(cudaMemsetAsync(first_inside, 0xff, sizeof(unsigned long long), c->stream));
  BIE_TRY(launch_foot_points(c, xobs, M, foot_elem, foot, first_inside));
  unsigned long long bad = ~0ull;
  BIE_CUDA_TRY(cudaMemcpyAsync(&bad, first_inside, sizeof(bad), cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (bad != ~0ull)
    return fail(BIE_ERR_INVALID_ARG, "observation point " + std::to_string(bad) +
                                         " lies inside a scatterer (Eq. BRIEFdmn needs points in the fluid)");
  const int64_t Ns = c->lin_N > 0 ? c->lin_N : c->N;  // nodes of the caller's surface values
  if (c->lin_N > 0) BIE_TRY(ensure_buf(c, c->work5, (size_t)kb * 2 * c->N * sizeof(cd)));
  for (int64_t k0 = 0; k0 < Nk; k0 += kb) {
    const int nk = (int)std::min<int64_t>(kb, Nk - k0);
    BIE_CUDA_TRY(cudaMemcpyAsync(kdev, k + k0, nk * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    const cd* s = (const cd*)surf + k0 * 2 * Ns;
    if (c->lin_N > 0) {  // linear elements: interpolate onto the flat quadratic image
      BIE_TRY(expand_linear(c, s, nk, (cd*)c->work5.p));
      s = (const cd*)c->work5.p;
    }
    cd* T = (cd*)T_out + k0 * M;
    if (mode == BIE_MODE_FP64)
      BIE_TRY(field64(c, kdev, nk, s, xobs, M, foot_elem, foot, T, scratch));
    else
      BIE_TRY(field_mixed(c, kdev, nk, s, xobs, M, foot_elem, foot, T, scratch, kb * perk));
  }
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

int bie_pulse_spectrum(bie_ctx* c, const double* s, int64_t P, int64_t Nt, void* S_out) {
  BIE_TRY(check_ctx(c, false));
  if (P < 0 || Nt < 2 || Nt > 4096 || (Nt & (Nt - 1)))
    return fail(BIE_ERR_INVALID_ARG, "Nt must be a power of two in [2, 4096] and P >= 0");
  if (P == 0) return BIE_OK;
  if (!s || !S_out) return fail(BIE_ERR_INVALID_ARG, "NULL pointer");
  BIE_TRY(pulse_spectrum(c, s, P, (int)Nt, (cd*)S_out));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

int bie_synthesize(bie_ctx* c, const void* T, const int64_t* midx, int64_t Nk, int64_t M, const void* S, int64_t P,
                   int64_t Nt, void* out, int out_dtype) {
  BIE_TRY(check_ctx(c, false));
  if (P < 0 || M < 0 || Nk < 0 || Nt < 2 || Nt > 4096 || (Nt & (Nt - 1)))
    return fail(BIE_ERR_INVALID_ARG, "need P, M, Nk >= 0 and Nt a power of two in [2, 4096]");
  if (out_dtype != 0 && out_dtype != 1) return fail(BIE_ERR_INVALID_ARG, "out_dtype must be 0 (f64) or 1 (f32)");
  if (P > 65535) return fail(BIE_ERR_INVALID_ARG, "P > 65535");
  if (P == 0 || M == 0) return BIE_OK;
  if ((Nk > 0 && (!T || !midx)) || !S || !out) return fail(BIE_ERR_INVALID_ARG, "NULL pointer");
  for (int64_t r = 0; r < Nk; ++r) {
    if (midx[r] < 0 || midx[r] > Nt / 2) return fail(BIE_ERR_INVALID_ARG, "midx out of [0, Nt/2]");
    if (r > 0 && midx[r] <= midx[r - 1]) return fail(BIE_ERR_INVALID_ARG, "midx must be strictly increasing");
  }
  BIE_TRY(ensure_buf(c, c->work3, (size_t)std::max<int64_t>(Nk, 1) * sizeof(int64_t)));
  int64_t* md = (int64_t*)c->work3.p;
  if (Nk > 0) BIE_CUDA_TRY(cudaMemcpyAsync(md, midx, Nk * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  BIE_TRY(synthesize(c, (const cd*)T, md, (int)Nk, M, (const cd*)S, P, (int)Nt, out, out_dtype));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

int bie_top_frequencies(bie_ctx* c, const void* S, int64_t P, int64_t Nt, int64_t K, int64_t* midx_out) {
  BIE_TRY(check_ctx(c, false));
  if (P < 1 || Nt < 2 || Nt > 4096 || (Nt & (Nt - 1)))
    return fail(BIE_ERR_INVALID_ARG, "need P >= 1 and Nt a power of two in [2, 4096]");
  const int64_t nm = Nt / 2 + 1;
  if (K < 0 || K > nm) return fail(BIE_ERR_INVALID_ARG, "K must be in [0, Nt/2 + 1]");
  if (K == 0) return BIE_OK;
  if (!S || !midx_out) return fail(BIE_ERR_INVALID_ARG, "NULL pointer");
  BIE_TRY(ensure_buf(c, c->work3, (size_t)K * sizeof(int64_t)));
  int64_t* md = (int64_t*)c->work3.p;
  BIE_TRY(top_frequencies(c, (const cd*)S, P, (int)nm, (int)K, md));
  BIE_CUDA_TRY(cudaMemcpyAsync(midx_out, md, (size_t)K * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

int bie_solve_frequencies_multi(bie_ctx* c, const double* k, int64_t Nk, const double* dirs, int64_t ndir, int mode,
                                void* surf_out, bie_report* rep) {
  BIE_TRY(check_ctx(c, true));
  BIE_TRY(check_k(k, Nk));
  if (ndir < 1 || ndir > 4096) return fail(BIE_ERR_INVALID_ARG, "ndir must be in [1, 4096]");
  if (!dirs) return fail(BIE_ERR_INVALID_ARG, "NULL dirs");
  std::vector<double> d(3 * ndir);
  for (int64_t i = 0; i < ndir; ++i) {
    const double* v = dirs + 3 * i;
    const double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(n > 0.0) || !std::isfinite(n))
      return fail(BIE_ERR_INVALID_ARG, "direction " + std::to_string(i) + " must be finite and non-zero");
    for (int t = 0; t < 3; ++t) d[3 * i + t] = v[t] / n;
  }
  if (Nk == 0) return BIE_OK;
  if (!surf_out) return fail(BIE_ERR_INVALID_ARG, "NULL surf_out");
  if (c->lin_N > 0) return fail(BIE_ERR_INVALID_ARG, "linear elements: one direction per call (bie_solve_frequencies)");
  if (mode == BIE_MODE_FP64) return solve_fp64_multi(c, k, Nk, d.data(), (int)ndir, (cd*)surf_out, rep);
  if (mode == BIE_MODE_MIXED)
    return solve_mixed(c, k, Nk, (cd*)surf_out, rep, nullptr, nullptr, nullptr, d.data(), (int)ndir);
  return fail(BIE_ERR_INVALID_ARG, "bie_solve_frequencies_multi supports BIE_MODE_FP64 and BIE_MODE_MIXED");
}

}  // extern "C"
