// synth.cu -- pulse spectra and space-time synthesis by the discrete Fourier transform with the
// sign of Eq. (inverseFourier) (exp(-i omega t)), evaluated by a radix-2 FFT (the last paragraph
// of Sec. 3 asks for the discrete fast Fourier transform).
//   spectrum:  S[p][m] = sum_n s[p][n] exp(+2 pi i m n / Nt) = conj(FFT(s))_m  (real s)
//   synthesis: out[p][x][n] = (1/Nt) Re sum_m c_m exp(-2 pi i m n / Nt),  c_m = w_m S[p][m] T[m][x],
//              w_0 = w_{Nt/2} = 1, else 2 (the m > Nt/2 half is the complex conjugate).
// One CTA transforms one signal in shared memory with a Stockham (self-sorting) radix-2 FFT.
#include <mutex>

#include "bie_common.cuh"

namespace bie {

template <class S> struct C2 { S re, im; };

// tw[j] = exp(-2 pi i j / n), j < n/2, from sincospi (correctly rounded to ~1 ulp in FP64).
__global__ void k_twiddles(int n, double2* tw) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n / 2) return;
  double s, c;
  sincospi(2.0 * (double)j / (double)n, &s, &c);
  tw[j] = make_double2(c, -s);
}

// Forward FFT of buf (length n, power of two) in place, using tmp as the ping-pong partner.
// Returns the buffer that holds the result.
template <class S>
__device__ C2<S>* stockham(C2<S>* buf, C2<S>* tmp, int n, const double2* __restrict__ tw) {
  C2<S>* x = buf;
  C2<S>* y = tmp;
  for (int m = 1; m < n; m <<= 1) {
    const int twstep = n / (2 * m);
    for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
      const int j = t / m, kk = t - j * m;
      const double2 w2 = tw[kk * twstep];
      const C2<S> w = {(S)w2.x, (S)w2.y};
      const C2<S> a = x[j * m + kk], b = x[j * m + kk + n / 2];
      const C2<S> wb = {w.re * b.re - w.im * b.im, w.re * b.im + w.im * b.re};
      y[2 * j * m + kk] = {a.re + wb.re, a.im + wb.im};
      y[2 * j * m + kk + m] = {a.re - wb.re, a.im - wb.im};
    }
    __syncthreads();
    C2<S>* t = x;
    x = y;
    y = t;
  }
  return x;
}

template <class S>
__global__ void k_pulse_spectrum(const double* __restrict__ s, int n, const double2* __restrict__ tw,
                                 cd* __restrict__ Sout) {
  extern __shared__ unsigned char smem_raw[];
  C2<S>* buf = reinterpret_cast<C2<S>*>(smem_raw);
  C2<S>* tmp = buf + n;
  const double* sp = s + (int64_t)blockIdx.x * n;
  for (int t = threadIdx.x; t < n; t += blockDim.x) buf[t] = {(S)sp[t], (S)0};
  __syncthreads();
  C2<S>* X = stockham<S>(buf, tmp, n, tw);
  cd* o = Sout + (int64_t)blockIdx.x * (n / 2 + 1);
  for (int t = threadIdx.x; t <= n / 2; t += blockDim.x) o[t] = {(double)X[t].re, -(double)X[t].im};
}

// grid: (M, P); one signal per CTA.
template <class S, class O>
__global__ void k_synth(const cd* __restrict__ T, const int64_t* __restrict__ midx, int nk, int64_t M,
                        const cd* __restrict__ Sp, int n, const double2* __restrict__ tw, O* __restrict__ out) {
  extern __shared__ unsigned char smem_raw[];
  C2<S>* buf = reinterpret_cast<C2<S>*>(smem_raw);
  C2<S>* tmp = buf + n;
  const int64_t x = blockIdx.x;
  const int p = blockIdx.y;
  for (int t = threadIdx.x; t < n; t += blockDim.x) buf[t] = {(S)0, (S)0};
  __syncthreads();
  const cd* Srow = Sp + (int64_t)p * (n / 2 + 1);
  for (int r = threadIdx.x; r < nk; r += blockDim.x) {
    const int m = (int)midx[r];
    const double w = (m == 0 || 2 * m == n) ? 1.0 : 2.0;
    const cd a = cmul(Srow[m], T[(int64_t)r * M + x]);
    buf[m] = {(S)(w * a.re), (S)(w * a.im)};
  }
  __syncthreads();
  C2<S>* X = stockham<S>(buf, tmp, n, tw);
  O* o = out + ((int64_t)p * M + x) * n;
  const S inv = (S)1 / (S)n;
  for (int t = threadIdx.x; t < n; t += blockDim.x) o[t] = (O)(X[t].re * inv);
}

static int twiddle_table(bie_ctx* c, int n, double2** tw) {
  BIE_TRY(ensure_buf(c, c->work2, (size_t)(n / 2 + 1) * sizeof(double2)));
  *tw = (double2*)c->work2.p;
  BIE_LAUNCH(k_twiddles<<<(n / 2 + 255) / 256, 256, 0, c->stream>>>(n, *tw));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int pulse_spectrum(bie_ctx* c, const double* s, int64_t P, int n, cd* Sout) {
  double2* tw;
  BIE_TRY(twiddle_table(c, n, &tw));
  size_t smem = 2 * (size_t)n * sizeof(C2<double>);
  BIE_TRY((set_smem_max(k_pulse_spectrum<double>)));
  BIE_LAUNCH(k_pulse_spectrum<double><<<(unsigned)P, std::min(512, n / 2), smem, c->stream>>>(s, n, tw, Sout));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int synthesize(bie_ctx* c, const cd* T, const int64_t* midx_dev, int nk, int64_t M, const cd* Sp, int64_t P, int n,
               void* out, int out_dtype) {
  double2* tw;
  BIE_TRY(twiddle_table(c, n, &tw));
  dim3 g((unsigned)M, (unsigned)P);
  int threads = std::min(512, std::max(32, n / 2));
  if (out_dtype == 0) {
    size_t smem = 2 * (size_t)n * sizeof(C2<double>);
    BIE_TRY((set_smem_max(k_synth<double, double>)));
    BIE_LAUNCH(k_synth<double, double><<<g, threads, smem, c->stream>>>(T, midx_dev, nk, M, Sp, n, tw, (double*)out));
  } else {
    size_t smem = 2 * (size_t)n * sizeof(C2<float>);
    BIE_TRY((set_smem_max(k_synth<float, float>)));
    BIE_LAUNCH(k_synth<float, float><<<g, threads, smem, c->stream>>>(T, midx_dev, nk, M, Sp, n, tw, (float*)out));
  }
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

// ------------------------------------------------------------------------------------------
// Dominant frequencies (Sec. 4, Table I; Sec. 5): the space-time field is accurate already from
// the wavenumbers at which the incident spectrum is largest, so only those need a frequency
// solve.  One CTA ranks m = 0 .. nm-1 by max over the pulses of |S[p][m]|^2 (ties: the lower m
// first) with a bitonic sort in shared memory, keeps the first K and sorts them ascending.
// ------------------------------------------------------------------------------------------
constexpr int kTopMax = 4096;  // padded sort length (nm = Nt/2 + 1 <= 2049)

__global__ void __launch_bounds__(1024) k_top_frequencies(const cd* __restrict__ S, int64_t P, int nm, int K,
                                                          int64_t* __restrict__ midx_out) {
  extern __shared__ unsigned char smem_raw[];
  double* key = reinterpret_cast<double*>(smem_raw);     // [kTopMax]
  int32_t* idx = reinterpret_cast<int32_t*>(key + kTopMax);  // [kTopMax]
  int L = 1;
  while (L < nm) L <<= 1;
  for (int m = threadIdx.x; m < L; m += blockDim.x) {
    double a = -1.0;  // padding sorts last
    if (m < nm) {
      a = 0.0;
      for (int64_t p = 0; p < P; ++p) {
        const cd v = S[p * nm + m];
        a = fmax(a, v.re * v.re + v.im * v.im);
      }
    }
    key[m] = a;
    idx[m] = m;
  }
  __syncthreads();
  // descending by key, ascending by index on ties
  for (int size = 2; size <= L; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < L / 2; t += blockDim.x) {
        const int i = 2 * t - (t & (stride - 1)), j = i + stride;
        const bool up = (i & size) == 0;  // this run ends in the wanted order
        const bool j_first = key[j] > key[i] || (key[j] == key[i] && idx[j] < idx[i]);
        if (j_first == up) {
          const double tk = key[i]; key[i] = key[j]; key[j] = tk;
          const int32_t ti = idx[i]; idx[i] = idx[j]; idx[j] = ti;
        }
      }
      __syncthreads();
    }
  // the K selected indices in ascending order
  int LK = 1;
  while (LK < K) LK <<= 1;
  for (int t = threadIdx.x; t < LK; t += blockDim.x) key[t] = t < K ? (double)idx[t] : 1e300;
  __syncthreads();
  for (int size = 2; size <= LK; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < LK / 2; t += blockDim.x) {
        const int i = 2 * t - (t & (stride - 1)), j = i + stride;
        const bool up = (i & size) == 0;
        if ((key[j] < key[i]) == up) {
          const double tk = key[i]; key[i] = key[j]; key[j] = tk;
        }
      }
      __syncthreads();
    }
  for (int t = threadIdx.x; t < K; t += blockDim.x) midx_out[t] = (int64_t)key[t];
}

int top_frequencies(bie_ctx* c, const cd* S, int64_t P, int nm, int K, int64_t* midx_dev) {
  if (nm > kTopMax) return fail(BIE_ERR_INVALID_ARG, "too many frequencies to rank");
  const size_t smem = kTopMax * (sizeof(double) + sizeof(int32_t));
  BIE_TRY((set_smem_max(k_top_frequencies)));
  BIE_LAUNCH(k_top_frequencies<<<1, 1024, smem, c->stream>>>(S, P, nm, K, midx_dev));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

// ------------------------------------------------------------------------------------------
// Allocation-free synthesis.  Some callers cannot allocate device memory while they run: a host
// framework that hands out a fixed device-memory budget through its own pool, or a latency-bound
// pipeline in which cudaMalloc/cudaFree would synchronise the device.  For them the synthesis's
// scratch (the FFT twiddle table and the device copy of the frequency indices) lives in one
// file-scope device array instead of context buffers, and no context is needed.
// ------------------------------------------------------------------------------------------
constexpr size_t kNoAllocScratchBytes = 64 * 1024;  // twiddles <= 32 KB (Nt <= 4096) + indices <= 32 KB
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the array on the current device, looked up once per device (the host-side
// name of a __device__ variable is not a device address).
static int noalloc_scratch(void** out) {
  int dev = 0;
  BIE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(BIE_ERR_INVALID_ARG, "device index too large");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return BIE_OK;
}

}  // namespace bie

extern "C" int bie_synthesize_noalloc(const void* T, const int64_t* midx, int64_t Nk, int64_t M, const void* S,
                                      int64_t P, int64_t Nt, void* out, int out_dtype, void* stream) {
  using namespace bie;
  if (P < 0 || M < 0 || Nk < 0 || Nt < 2 || Nt > 4096 || (Nt & (Nt - 1)))
    return fail(BIE_ERR_INVALID_ARG, "need P, M, Nk >= 0 and Nt a power of two in [2, 4096]");
  if (out_dtype != 0 && out_dtype != 1) return fail(BIE_ERR_INVALID_ARG, "out_dtype must be 0 (f64) or 1 (f32)");
  if (P > 65535) return fail(BIE_ERR_INVALID_ARG, "P > 65535");
  if ((size_t)Nk * sizeof(int64_t) > kNoAllocScratchBytes / 2)
    return fail(BIE_ERR_INVALID_ARG, "Nk = " + std::to_string(Nk) + " exceeds the fixed scratch (at most " +
                                         std::to_string(kNoAllocScratchBytes / 2 / sizeof(int64_t)) + ")");
  if (P == 0 || M == 0) return BIE_OK;
  if ((Nk > 0 && (!T || !midx)) || !S || !out) return fail(BIE_ERR_INVALID_ARG, "NULL pointer");
  for (int64_t r = 0; r < Nk; ++r) {
    if (midx[r] < 0 || midx[r] > Nt / 2) return fail(BIE_ERR_INVALID_ARG, "midx out of [0, Nt/2]");
    if (r > 0 && midx[r] <= midx[r - 1]) return fail(BIE_ERR_INVALID_ARG, "midx must be strictly increasing");
  }
  void* base = nullptr;
  BIE_TRY(noalloc_scratch(&base));
  cudaStream_t st = (cudaStream_t)stream;
  const int n = (int)Nt;
  double2* tw = (double2*)base;  // n/2 entries, rewritten by every call
  int64_t* md = (int64_t*)((char*)base + kNoAllocScratchBytes / 2);
  if (Nk > 0) BIE_CUDA_TRY(cudaMemcpyAsync(md, midx, Nk * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  BIE_LAUNCH(k_twiddles<<<(n / 2 + 255) / 256, 256, 0, st>>>(n, tw));
  dim3 g((unsigned)M, (unsigned)P);
  const int threads = std::min(512, std::max(32, n / 2));
  if (out_dtype == 0) {
    const size_t smem = 2 * (size_t)n * sizeof(C2<double>);
    BIE_TRY((set_smem_max(k_synth<double, double>)));
    BIE_LAUNCH(k_synth<double, double><<<g, threads, smem, st>>>((const cd*)T, md, (int)Nk, M, (const cd*)S, n, tw, (double*)out));
  } else {
    const size_t smem = 2 * (size_t)n * sizeof(C2<float>);
    BIE_TRY((set_smem_max(k_synth<float, float>)));
    BIE_LAUNCH(k_synth<float, float><<<g, threads, smem, st>>>((const cd*)T, md, (int)Nk, M, (const cd*)S, n, tw, (float*)out));
  }
  BIE_CUDA_TRY(cudaGetLastError());
  // the host index array must outlive its asynchronous copy
  BIE_CUDA_TRY(cudaStreamSynchronize(st));
  return BIE_OK;
}
